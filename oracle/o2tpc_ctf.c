/*
 * o2tpc_ctf.c - oracle of the compressed Time Frame (CTF): hit removal,
 * track-model compression and rANS entropy coding of the TPC clusters.
 *
 * TEST INFRASTRUCTURE ONLY (see o2tpc_oracle.h).  Plain C, single thread; it
 * shares no code with the CUDA path.
 *
 * Sec. 2.2: TPC clusters are the bulk of the stored data; hits of tracks not
 * used for physics are removed, the remaining hits go through entropy
 * reduction (track-model compression), and a lossless ANS entropy coder is
 * the last stage.  The paper gives no formats or parameters; this file fixes
 * them (the readings):
 *
 *  removal   clusters of tracks with pT < 0.1 GeV (|q/pT| > 10 / GeV) are
 *            dropped; all other clusters are kept;
 *  order     kept tracks ordered by the input index of their first cluster,
 *            each with its clusters in track order; then every cluster on no
 *            track, in the sorted-hit order (TF, sector, row, cell, input);
 *  fields    per cluster: sector delta to the previous cluster of the
 *            sequence (mod 36), row delta (mod 256), y and zeta residuals in
 *            the integer cluster units (y 1/160 cm, zeta 1/64 time bin);
 *            a track cluster with two predecessors in its own sector segment
 *            takes as residual v - pred, pred = v1 + floor((v1 - v0)(r - r1)
 *            / (r1 - r0)) from those two (a straight-line track model in
 *            integer arithmetic, so a decoder repeats it exactly); any other
 *            cluster the difference to the previous cluster of the sequence;
 *            residuals zigzag-mapped, y to 16 and zeta to 32 bits; per kept
 *            track its cluster count (16 bits);
 *  streams   the fields split into ten byte planes: sector, row, y lo/hi,
 *            zeta bytes 0-3, count lo/hi;
 *  rANS      per stream a static table of 256 frequencies summing to 4096
 *            (counts scaled down with floor, at least 1 for a present
 *            symbol; the surplus or deficit goes to the largest entries,
 *            ties to the lower symbol); chunks of 4096 symbols, each coded
 *            independently (32-bit state in [2^23, 2^31), byte-wise
 *            renormalisation, symbols coded last to first; a chunk is its
 *            final state, 4 bytes little endian, followed by the emitted
 *            bytes in decoding order).
 *
 * Blob layout (little endian):
 *   u32 magic 'O2CT', u32 version 1, u32 n_tracks, u32 n_track_clusters,
 *   u32 n_unattached, u32 n_streams (10);
 *   per stream: u32 n_symbols, u32 n_chunks, u16 freq[256], u32 chunk_bytes[n_chunks];
 *   then the chunk payloads, stream by stream, chunk by chunk.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "o2tpc_oracle.h"

#define C_SCALE_BITS 12
#define C_M (1u << C_SCALE_BITS)
#define C_L (1u << 23)
#define C_CHUNK 4096
#define C_NSTREAM 10
#define C_NROW 152

void oracle_buffer_free(void* p) { free(p); }

/* ---------------------------------------------------------------- tables */
void oracle_ctf_normalize(const uint64_t* count, uint16_t* freq) {
  uint64_t n = 0;
  for (int s = 0; s < 256; ++s) n += count[s];
  memset(freq, 0, 256 * sizeof(uint16_t));
  if (n == 0) return;
  int64_t sum = 0;
  for (int s = 0; s < 256; ++s) {
    if (!count[s]) continue;
    uint64_t f = count[s] * (uint64_t)C_M / n;
    if (f < 1) f = 1;
    freq[s] = (uint16_t)f;
    sum += (int64_t)f;
  }
  int64_t d = (int64_t)C_M - sum;
  while (d != 0) {
    /* the largest entry (lowest symbol on ties) absorbs the difference, as far
     * as it can stay >= 1 */
    int best = -1;
    for (int s = 0; s < 256; ++s)
      if (freq[s] && (best < 0 || freq[s] > freq[best])) best = s;
    if (d > 0) {
      freq[best] = (uint16_t)(freq[best] + d);
      d = 0;
    } else {
      int64_t take = (int64_t)freq[best] - 1;
      if (take > -d) take = -d;
      freq[best] = (uint16_t)(freq[best] - take);
      d += take;
    }
  }
}

/* ------------------------------------------------------------------ rANS */
/* Codes sym[0, n) with the table; writes the chunk to out (capacity cap),
 * returns its byte count. */
static int64_t c_rans_chunk(const uint8_t* sym, int64_t n, const uint16_t* freq, const uint32_t* cum, uint8_t* out,
                            int64_t cap) {
  uint8_t* buf = (uint8_t*)malloc((size_t)(2 * n + 16));
  int64_t p = 2 * n + 16; /* emitted bytes go backwards from the end */
  uint32_t x = C_L;
  for (int64_t i = n - 1; i >= 0; --i) {
    uint32_t f = freq[sym[i]], c = cum[sym[i]];
    uint32_t xmax = ((C_L >> C_SCALE_BITS) << 8) * f;
    while (x >= xmax) {
      buf[--p] = (uint8_t)(x & 0xff);
      x >>= 8;
    }
    x = ((x / f) << C_SCALE_BITS) + (x % f) + c;
  }
  int64_t nb = 4 + (2 * n + 16 - p);
  if (nb <= cap) {
    out[0] = (uint8_t)x; out[1] = (uint8_t)(x >> 8); out[2] = (uint8_t)(x >> 16); out[3] = (uint8_t)(x >> 24);
    memcpy(out + 4, buf + p, (size_t)(nb - 4));
  }
  free(buf);
  return nb;
}

static int c_rans_decode_chunk(const uint8_t* in, int64_t bytes, int64_t n, const uint16_t* freq, const uint32_t* cum,
                               const uint8_t* slot2sym, uint8_t* sym) {
  if (bytes < 4) return -1;
  uint32_t x = (uint32_t)in[0] | ((uint32_t)in[1] << 8) | ((uint32_t)in[2] << 16) | ((uint32_t)in[3] << 24);
  int64_t p = 4;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t slot = x & (C_M - 1);
    uint8_t s = slot2sym[slot];
    sym[i] = s;
    x = freq[s] * (x >> C_SCALE_BITS) + slot - cum[s];
    while (x < C_L) {
      if (p >= bytes) return -1;
      x = (x << 8) | in[p++];
    }
  }
  return (p == bytes && x == C_L) ? 0 : -1;
}

/* Codes a whole stream: table, chunk sizes and payloads appended to *blob. */
typedef struct { uint8_t* p; int64_t n, cap; } c_buf;
static void c_put(c_buf* b, const void* src, int64_t n) {
  if (n <= 0) return;
  while (b->n + n > b->cap) { b->cap = b->cap ? 2 * b->cap : 4096; b->p = (uint8_t*)realloc(b->p, (size_t)b->cap); }
  memcpy(b->p + b->n, src, (size_t)n);
  b->n += n;
}
static void c_put32(c_buf* b, uint32_t v) {
  uint8_t t[4] = {(uint8_t)v, (uint8_t)(v >> 8), (uint8_t)(v >> 16), (uint8_t)(v >> 24)};
  c_put(b, t, 4);
}
static void c_put16(c_buf* b, uint16_t v) {
  uint8_t t[2] = {(uint8_t)v, (uint8_t)(v >> 8)};
  c_put(b, t, 2);
}

static void c_code_stream(const uint8_t* sym, int64_t n, c_buf* head, c_buf* body) {
  uint64_t count[256] = {0};
  for (int64_t i = 0; i < n; ++i) count[sym[i]]++;
  uint16_t freq[256];
  uint32_t cum[257];
  oracle_ctf_normalize(count, freq);
  cum[0] = 0;
  for (int s = 0; s < 256; ++s) cum[s + 1] = cum[s] + freq[s];
  int64_t nch = (n + C_CHUNK - 1) / C_CHUNK;
  c_put32(head, (uint32_t)n);
  c_put32(head, (uint32_t)nch);
  for (int s = 0; s < 256; ++s) c_put16(head, freq[s]);
  uint8_t* tmp = (uint8_t*)malloc((size_t)(2 * C_CHUNK + 16));
  for (int64_t c = 0; c < nch; ++c) {
    int64_t a = c * C_CHUNK, m = (n - a < C_CHUNK) ? n - a : C_CHUNK;
    int64_t nb = c_rans_chunk(sym + a, m, freq, cum, tmp, 2 * C_CHUNK + 16);
    c_put32(head, (uint32_t)nb);
    c_put(body, tmp, nb);
  }
  free(tmp);
}

int64_t oracle_rans_encode(const uint8_t* sym, int64_t n, uint8_t** out) {
  c_buf h = {0}, b = {0};
  c_code_stream(sym, n, &h, &b);
  c_put(&h, b.p, b.n);
  free(b.p);
  *out = h.p;
  return h.n;
}

static uint32_t c_get32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

/* Decodes one stream whose header starts at *hp and whose payloads start at
 * *bp; advances both.  Returns the symbol count, -1 on a malformed stream. */
static int64_t c_decode_stream(const uint8_t** hp, const uint8_t* hend, const uint8_t** bp, const uint8_t* bend,
                               uint8_t** symOut) {
  const uint8_t* h = *hp;
  if (hend - h < 8 + 512) return -1;
  int64_t n = c_get32(h), nch = c_get32(h + 4);
  h += 8;
  uint16_t freq[256];
  uint32_t cum[257];
  cum[0] = 0;
  for (int s = 0; s < 256; ++s) { freq[s] = (uint16_t)(h[2 * s] | (h[2 * s + 1] << 8)); cum[s + 1] = cum[s] + freq[s]; }
  h += 512;
  if (nch != (n + C_CHUNK - 1) / C_CHUNK || (n > 0 && cum[256] != C_M) || hend - h < 4 * nch) return -1;
  uint8_t slot2sym[C_M];
  for (int s = 0; s < 256; ++s) for (uint32_t k = cum[s]; k < cum[s + 1] && k < C_M; ++k) slot2sym[k] = (uint8_t)s;
  uint8_t* sym = (uint8_t*)malloc((size_t)n + 1);
  const uint8_t* b = *bp;
  for (int64_t c = 0; c < nch; ++c) {
    int64_t nb = c_get32(h + 4 * c);
    int64_t a = c * C_CHUNK, m = (n - a < C_CHUNK) ? n - a : C_CHUNK;
    if (bend - b < nb || c_rans_decode_chunk(b, nb, m, freq, cum, slot2sym, sym + a) != 0) { free(sym); return -1; }
    b += nb;
  }
  *hp = h + 4 * nch;
  *bp = b;
  *symOut = sym;
  return n;
}

int64_t oracle_rans_decode(const uint8_t* blob, int64_t bytes, uint8_t** out) {
  const uint8_t* h = blob;
  if (bytes < 8) return -1;
  int64_t nch = c_get32(blob + 4);
  const uint8_t* body = blob + 8 + 512 + 4 * nch;
  if (body > blob + bytes) return -1;
  return c_decode_stream(&h, body, &body, blob + bytes, out);
}

/* -------------------------------------------------------------- the CTF */
static int64_t c_fdiv(int64_t a, int64_t b) { /* floor division, b > 0 */
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

/* Residual of value v for sequence position i (see the header). */
static int64_t c_pred(int has2, int64_t r0, int64_t v0, int64_t r1, int64_t v1, int64_t r, int64_t prev) {
  if (!has2) return prev;
  return v1 + c_fdiv((v1 - v0) * (r - r1), r1 - r0);
}

int64_t oracle_ctf_encode(int64_t n_clusters, const int32_t* sector, const int32_t* row, const int32_t* y,
                          const int32_t* z, int64_t n_tracks, const int64_t* trk_off, const int32_t* trk_cl,
                          const double* trk_qpt, const int32_t* sorted_orig, int64_t n_sorted, uint8_t** out) {
  /* kept tracks by the input index of their first cluster */
  int8_t* onTrack = (int8_t*)calloc((size_t)n_clusters + 1, 1);
  int32_t* firstOf = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n_clusters + 1));
  for (int64_t i = 0; i < n_clusters; ++i) firstOf[i] = -1;
  int64_t nKeptTrk = 0, nTrkCl = 0;
  for (int64_t t = 0; t < n_tracks; ++t) {
    for (int64_t q = trk_off[t]; q < trk_off[t + 1]; ++q) onTrack[trk_cl[q]] = 1;
    if (trk_off[t + 1] == trk_off[t] || !(trk_qpt[t] >= -10.0 && trk_qpt[t] <= 10.0)) continue; /* removed */
    firstOf[trk_cl[trk_off[t]]] = (int32_t)t;
    ++nKeptTrk;
    nTrkCl += trk_off[t + 1] - trk_off[t];
  }
  int64_t nUn = 0;
  for (int64_t s = 0; s < n_sorted; ++s) nUn += !onTrack[sorted_orig[s]];
  int64_t nSeq = nTrkCl + nUn;
  uint8_t* st[C_NSTREAM];
  int64_t len[C_NSTREAM] = {nSeq, nSeq, nSeq, nSeq, nSeq, nSeq, nSeq, nSeq, nKeptTrk, nKeptTrk};
  for (int k = 0; k < C_NSTREAM; ++k) st[k] = (uint8_t*)malloc((size_t)len[k] + 1);
  int64_t o = 0, ot = 0;
  int32_t ps = 0, pr = 0, py = 0, pz = 0; /* previous cluster of the sequence */
#define C_EMIT(sec, rw, yy, zz, has2, r0, y0, z0, r1, y1, z1)                                           \
  do {                                                                                                  \
    int64_t ry = (int64_t)(yy) - c_pred(has2, r0, y0, r1, y1, rw, py);                                  \
    int64_t rz = (int64_t)(zz) - c_pred(has2, r0, z0, r1, z1, rw, pz);                                  \
    int16_t ry16 = (int16_t)(uint16_t)(uint64_t)ry;                                                     \
    int32_t rz32 = (int32_t)(uint32_t)(uint64_t)rz;                                                     \
    uint16_t zy = (uint16_t)(((uint16_t)ry16 << 1) ^ (uint16_t)(ry16 >> 15));                           \
    uint32_t zzz = ((uint32_t)rz32 << 1) ^ (uint32_t)(rz32 >> 31);                                      \
    st[0][o] = (uint8_t)((((sec) - ps) % 36 + 36) % 36);                                                \
    st[1][o] = (uint8_t)(((rw) - pr) & 0xff);                                                           \
    st[2][o] = (uint8_t)zy; st[3][o] = (uint8_t)(zy >> 8);                                              \
    st[4][o] = (uint8_t)zzz; st[5][o] = (uint8_t)(zzz >> 8); st[6][o] = (uint8_t)(zzz >> 16);           \
    st[7][o] = (uint8_t)(zzz >> 24);                                                                    \
    ++o; ps = (sec); pr = (rw); py = (yy); pz = (zz);                                                   \
  } while (0)
  for (int64_t c = 0; c < n_clusters; ++c) {
    int32_t t = firstOf[c];
    if (t < 0) continue;
    int64_t m = trk_off[t + 1] - trk_off[t];
    st[8][ot] = (uint8_t)m; st[9][ot] = (uint8_t)(m >> 8); ++ot;
    for (int64_t q = 0; q < m; ++q) {
      int32_t h = trk_cl[trk_off[t] + q];
      int has2 = 0;
      int32_t h0 = 0, h1 = 0;
      if (q >= 2) {
        h0 = trk_cl[trk_off[t] + q - 2]; h1 = trk_cl[trk_off[t] + q - 1];
        has2 = sector[h0] == sector[h] && sector[h1] == sector[h] && row[h0] < row[h1] && row[h1] < row[h];
      }
      C_EMIT(sector[h], row[h], y[h], z[h], has2, row[h0], y[h0], z[h0], row[h1], y[h1], z[h1]);
    }
  }
  for (int64_t s = 0; s < n_sorted; ++s) {
    int32_t h = sorted_orig[s];
    if (onTrack[h]) continue;
    C_EMIT(sector[h], row[h], y[h], z[h], 0, 0, 0, 0, 0, 0, 0);
  }
#undef C_EMIT
  c_buf head = {0}, body = {0};
  c_put32(&head, 0x5443324Fu); /* 'O2CT' */
  c_put32(&head, 1);
  c_put32(&head, (uint32_t)nKeptTrk);
  c_put32(&head, (uint32_t)nTrkCl);
  c_put32(&head, (uint32_t)nUn);
  c_put32(&head, C_NSTREAM);
  for (int k = 0; k < C_NSTREAM; ++k) c_code_stream(st[k], len[k], &head, &body);
  c_put(&head, body.p, body.n);
  free(body.p);
  for (int k = 0; k < C_NSTREAM; ++k) free(st[k]);
  free(onTrack); free(firstOf);
  *out = head.p;
  return head.n;
}

int64_t oracle_ctf_decode(const uint8_t* blob, int64_t bytes, int32_t** sector, int32_t** row, int32_t** y,
                          int32_t** z, int64_t* n_tracks, int64_t** trk_len) {
  if (bytes < 24 || c_get32(blob) != 0x5443324Fu || c_get32(blob + 4) != 1 || c_get32(blob + 20) != C_NSTREAM)
    return -1;
  int64_t nT = c_get32(blob + 8), nTC = c_get32(blob + 12), nU = c_get32(blob + 16), nSeq = nTC + nU;
  /* the stream headers are laid out one after the other; the payloads follow
   * the last header */
  const uint8_t* h = blob + 24;
  const uint8_t* body = h;
  for (int k = 0; k < C_NSTREAM; ++k) {
    if (blob + bytes - body < 8) return -1;
    body += 8 + 512 + 4 * (int64_t)c_get32(body + 4);
  }
  if (body > blob + bytes) return -1;
  uint8_t* st[C_NSTREAM] = {0};
  int bad = 0;
  for (int k = 0; k < C_NSTREAM; ++k) {
    int64_t want = k < 8 ? nSeq : nT;
    int64_t got = bad ? -1 : c_decode_stream(&h, body, &body, blob + bytes, &st[k]);
    if (got != want) bad = 1;
  }
  if (bad) { for (int k = 0; k < C_NSTREAM; ++k) free(st[k]); return -1; }
  int32_t* S = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nSeq + 1));
  int32_t* R = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nSeq + 1));
  int32_t* Y = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nSeq + 1));
  int32_t* Z = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nSeq + 1));
  int64_t* L = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nT + 1));
  int32_t ps = 0, pr = 0, py = 0, pz = 0;
  int64_t o = 0;
  for (int64_t t = 0; t <= nT; ++t) {
    int64_t m = (t < nT) ? (int64_t)(st[8][t] | (st[9][t] << 8)) : nU; /* the unattached run last */
    if (t < nT) L[t] = m;
    int64_t begin = o;
    for (int64_t q = 0; q < m && o < nSeq; ++q, ++o) {
      int32_t sec = (ps + st[0][o]) % 36;
      int32_t rw = (pr + st[1][o]) & 0xff;
      uint16_t zy = (uint16_t)(st[2][o] | (st[3][o] << 8));
      uint32_t zzz = (uint32_t)st[4][o] | ((uint32_t)st[5][o] << 8) | ((uint32_t)st[6][o] << 16) |
                     ((uint32_t)st[7][o] << 24);
      int16_t ry = (int16_t)((zy >> 1) ^ (uint16_t)(-(int16_t)(zy & 1)));
      int32_t rz = (int32_t)((zzz >> 1) ^ (uint32_t)(-(int32_t)(zzz & 1)));
      int has2 = 0;
      if (t < nT && q >= 2) {
        int64_t a = o - 2, b = o - 1;
        has2 = S[a] == sec && S[b] == sec && R[a] < R[b] && R[b] < rw;
      }
      int64_t a = o - 2, b = o - 1;
      int64_t pyv = c_pred(has2, has2 ? R[a] : 0, has2 ? Y[a] : 0, has2 ? R[b] : 0, has2 ? Y[b] : 0, rw, py);
      int64_t pzv = c_pred(has2, has2 ? R[a] : 0, has2 ? Z[a] : 0, has2 ? R[b] : 0, has2 ? Z[b] : 0, rw, pz);
      int32_t yy = (int32_t)(int16_t)(uint16_t)(uint64_t)(pyv + ry);
      int32_t zz = (int32_t)(uint32_t)(uint64_t)(pzv + rz);
      S[o] = sec; R[o] = rw; Y[o] = yy; Z[o] = zz;
      ps = sec; pr = rw; py = yy; pz = zz;
    }
    (void)begin;
  }
  for (int k = 0; k < C_NSTREAM; ++k) free(st[k]);
  *sector = S; *row = R; *y = Y; *z = Z; *n_tracks = nT; *trk_len = L;
  return nSeq;
}
