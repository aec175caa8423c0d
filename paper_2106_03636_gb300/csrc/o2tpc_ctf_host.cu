// Host decoder of the compressed Time Frame written by csrc/k_ctf.cu: the
// reader side of the format (Sec. 2.2: the compressed TF is what is stored;
// decoding it must give back exactly the kept clusters).  Plain host code, no
// device work: a consumer of stored TFs needs no GPU.
//
// Format (see k_ctf.cu): header (magic 'O2CT', version 1, kept tracks, their
// clusters, other clusters, 10 streams), per stream (symbols, chunks,
// 256 frequencies summing to 4096, chunk sizes), then the chunk payloads.
// Each chunk holds at most 4096 symbols: a 32-bit rANS state (little endian)
// followed by the renormalisation bytes in decoding order.  The ten streams
// are byte planes of the per-cluster fields (sector delta mod 36, row delta
// mod 256, y residual lo/hi, zeta residual bytes 0-3) and of the per-track
// cluster counts (lo/hi); residuals are zigzag-mapped, against the straight
// line through the two previous clusters of the same sector segment of a
// track (rows ascending) or else against the previous cluster.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "o2tpc.h"

namespace {

constexpr uint32_t kMagic = 0x5443324Fu;
constexpr int kStreams = 10;
constexpr uint32_t kScaleBits = 12, kM = 1u << kScaleBits, kL = 1u << 23;
constexpr int64_t kChunk = 4096;
constexpr int kRows = 152;

uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

struct Reader {
  const uint8_t* p;
  uint64_t n, pos = 0;
  bool take(uint64_t k) { return pos + k <= n; }
};

// One stream: header at *h (advanced), payloads at *b (advanced).
bool decode_stream(Reader& h, Reader& b, std::vector<uint8_t>& out) {
  if (!h.take(8 + 512)) return false;
  const uint64_t nsym = rd32(h.p + h.pos), nch = rd32(h.p + h.pos + 4);
  h.pos += 8;
  uint32_t f[256], c[257];
  c[0] = 0;
  for (int s = 0; s < 256; ++s) {
    f[s] = (uint32_t)h.p[h.pos + 2 * s] | ((uint32_t)h.p[h.pos + 2 * s + 1] << 8);
    c[s + 1] = c[s] + f[s];
  }
  h.pos += 512;
  if (nch != (nsym + kChunk - 1) / kChunk || (nsym > 0 && c[256] != kM) || !h.take(4 * nch)) return false;
  std::vector<uint8_t> slot(kM);
  for (int s = 0; s < 256; ++s)
    for (uint32_t k = c[s]; k < c[s + 1] && k < kM; ++k) slot[k] = (uint8_t)s;
  out.assign(nsym, 0);
  for (uint64_t ch = 0; ch < nch; ++ch) {
    const uint64_t nb = rd32(h.p + h.pos + 4 * ch);
    if (nb < 4 || !b.take(nb)) return false;
    const uint8_t* q = b.p + b.pos;
    uint32_t x = rd32(q);
    uint64_t r = 4;
    const uint64_t a = ch * kChunk, m = (nsym - a < (uint64_t)kChunk) ? nsym - a : (uint64_t)kChunk;
    for (uint64_t i = 0; i < m; ++i) {
      const uint32_t sl = x & (kM - 1);
      const uint8_t s = slot[sl];
      out[a + i] = s;
      x = f[s] * (x >> kScaleBits) + sl - c[s];
      while (x < kL) {
        if (r >= nb) return false;
        x = (x << 8) | q[r++];
      }
    }
    if (r != nb || x != kL) return false;
    b.pos += nb;
  }
  h.pos += 4 * nch;
  return true;
}

long long floor_div(long long a, long long b) {  // b > 0
  long long q = a / b;
  if (a % b != 0 && a < 0) --q;
  return q;
}

}  // namespace

extern "C" int o2tpc_ctf_decode(const uint8_t* blob, uint64_t bytes, o2tpc_ctf_clusters* out) {
  if (!blob || !out) return O2TPC_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (bytes < 24 || rd32(blob) != kMagic || rd32(blob + 4) != 1 || rd32(blob + 20) != (uint32_t)kStreams)
    return O2TPC_EINVAL;
  const uint64_t nTrk = rd32(blob + 8), nTc = rd32(blob + 12), nFree = rd32(blob + 16), nSeq = nTc + nFree;
  // the headers come one after the other; the payloads follow the last
  Reader scan{blob, bytes, 24};
  for (int s = 0; s < kStreams; ++s) {
    if (!scan.take(8)) return O2TPC_EINVAL;
    const uint64_t nch = rd32(blob + scan.pos + 4);
    if (!scan.take(8 + 512 + 4 * nch)) return O2TPC_EINVAL;
    scan.pos += 8 + 512 + 4 * nch;
  }
  Reader h{blob, bytes, 24}, b{blob, bytes, scan.pos};
  std::vector<uint8_t> st[kStreams];
  try {
    for (int s = 0; s < kStreams; ++s) {
      if (!decode_stream(h, b, st[s])) return O2TPC_EINVAL;
      if (st[s].size() != (s < 8 ? nSeq : nTrk)) return O2TPC_EINVAL;
    }
    if (b.pos != bytes) return O2TPC_EINVAL;  // the payloads end the blob
  } catch (const std::bad_alloc&) {
    return O2TPC_ENOMEM;
  }
  int32_t* sec = static_cast<int32_t*>(std::malloc(4 * (nSeq + 1)));
  int32_t* row = static_cast<int32_t*>(std::malloc(4 * (nSeq + 1)));
  int32_t* y = static_cast<int32_t*>(std::malloc(4 * (nSeq + 1)));
  int32_t* z = static_cast<int32_t*>(std::malloc(4 * (nSeq + 1)));
  uint32_t* len = static_cast<uint32_t*>(std::malloc(4 * (nTrk + 1)));
  if (!sec || !row || !y || !z || !len) {
    std::free(sec), std::free(row), std::free(y), std::free(z), std::free(len);
    return O2TPC_ENOMEM;
  }
  int32_t ps = 0, pr = 0, py = 0, pz = 0;
  uint64_t o = 0, sumLen = 0;
  for (uint64_t t = 0; t <= nTrk; ++t) {
    const uint64_t m = t < nTrk ? ((uint64_t)st[8][t] | ((uint64_t)st[9][t] << 8)) : nFree;
    if (t < nTrk) {
      len[t] = (uint32_t)m;
      sumLen += m;
    }
    for (uint64_t q = 0; q < m; ++q, ++o) {
      if (o >= nSeq) break;
      const int32_t s = (ps + st[0][o]) % 36;
      const int32_t r = (pr + st[1][o]) & 0xff;
      const uint16_t zy = (uint16_t)(st[2][o] | (st[3][o] << 8));
      const uint32_t zz = (uint32_t)st[4][o] | ((uint32_t)st[5][o] << 8) | ((uint32_t)st[6][o] << 16) |
                          ((uint32_t)st[7][o] << 24);
      const int32_t ry = (int16_t)((zy >> 1) ^ (uint16_t)(0u - (zy & 1u)));
      const int32_t rz = (int32_t)((zz >> 1) ^ (0u - (zz & 1u)));
      // the straight line through the two previous clusters of the track's
      // current sector segment, else the previous cluster
      const bool two = t < nTrk && q >= 2 && sec[o - 2] == s && sec[o - 1] == s && row[o - 2] < row[o - 1] &&
                       row[o - 1] < r;
      long long predY = py, predZ = pz;
      if (two) {
        const long long r0 = row[o - 2], r1 = row[o - 1];
        predY = y[o - 1] + floor_div((long long)(y[o - 1] - y[o - 2]) * (r - r1), r1 - r0);
        predZ = z[o - 1] + floor_div((long long)(z[o - 1] - z[o - 2]) * (r - r1), r1 - r0);
      }
      sec[o] = s;
      row[o] = r;
      y[o] = (int32_t)(int16_t)(uint16_t)(uint64_t)(predY + ry);
      z[o] = (int32_t)(uint32_t)(uint64_t)(predZ + rz);
      ps = s;
      pr = r;
      py = y[o];
      pz = z[o];
    }
  }
  if (sumLen != nTc || o != nSeq) {
    std::free(sec), std::free(row), std::free(y), std::free(z), std::free(len);
    return O2TPC_EINVAL;
  }
  for (uint64_t i = 0; i < nSeq; ++i)
    if (row[i] >= kRows) {
      std::free(sec), std::free(row), std::free(y), std::free(z), std::free(len);
      return O2TPC_EINVAL;
    }
  out->n = nSeq;
  out->n_tracks = nTrk;
  out->sector = sec;
  out->row = row;
  out->y = y;
  out->zeta = z;
  out->track_len = len;
  return O2TPC_OK;
}

extern "C" void o2tpc_ctf_free(o2tpc_ctf_clusters* c) {
  if (!c) return;
  std::free(const_cast<int32_t*>(c->sector));
  std::free(const_cast<int32_t*>(c->row));
  std::free(const_cast<int32_t*>(c->y));
  std::free(const_cast<int32_t*>(c->zeta));
  std::free(const_cast<uint32_t*>(c->track_len));
  std::memset(c, 0, sizeof(*c));
}

extern "C" int o2tpc_ctf_records(const o2tpc_ctf_clusters* c, void* records) {
  if (!c || (c->n > 0 && !records)) return O2TPC_EINVAL;
  // pads per row: floor(2 x_r tan(10 deg) / 0.4 cm), x_r = 85 + r 160/151 cm
  int npads[kRows];
  for (int r = 0; r < kRows; ++r)
    npads[r] = (int)std::floor(2.0 * (85.0 + r * 160.0 / 151.0) * std::tan(10.0 * 3.14159265358979323846 / 180.0) / 0.4);
  uint8_t* o = static_cast<uint8_t*>(records);
  for (uint64_t i = 0; i < c->n; ++i, o += 12) {
    const int r = c->row[i];
    const long long pad64 = (long long)c->y[i] + 32ll * npads[r];
    const long long t64 = c->zeta[i];
    if (r < 0 || r >= kRows || c->sector[i] < 0 || c->sector[i] >= 36 || pad64 < 0 || pad64 > 0xffff || t64 < 0 ||
        t64 >= (1ll << 30))
      return O2TPC_EINVAL;
    o[0] = (uint8_t)t64;
    o[1] = (uint8_t)(t64 >> 8);
    o[2] = (uint8_t)(t64 >> 16);
    o[3] = (uint8_t)(t64 >> 24);
    o[4] = (uint8_t)pad64;
    o[5] = (uint8_t)(pad64 >> 8);
    o[6] = o[7] = 0;  // charges are not stored
    o[8] = (uint8_t)r;
    o[9] = (uint8_t)c->sector[i];
    o[10] = o[11] = 0;
  }
  return O2TPC_OK;
}
