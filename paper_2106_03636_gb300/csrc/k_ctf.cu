// Compressed Time Frame (Sec. 2.2): hit removal, track-model compression and
// rANS entropy coding of each TF's clusters, on the device after tracking.
//
// Sec. 2.2 says that clusters of tracks not used for physics are removed,
// that the remaining clusters go through entropy-reducing steps such as the
// track-model compression, and that a lossless ANS coder is the last stage.
// The formats and parameters are this implementation's reading:
//  * removal: clusters of tracks with |q/pT| > 10 / GeV (pT < 0.1 GeV);
//  * cluster sequence: kept tracks by the input index of their first
//    cluster, each with its clusters in track order, then every cluster on
//    no track in sorted-hit order;
//  * fields per cluster: sector delta to the previous cluster (mod 36), row
//    delta (mod 256), y and zeta residuals in integer cluster units: against
//    the straight line through the two previous clusters of the same sector
//    segment of the track (v1 + floor((v1 - v0)(r - r1) / (r1 - r0)), exact
//    in integers so a decoder repeats it), else against the previous cluster
//    of the sequence; zigzag-mapped, 16 bits for y, 32 for zeta; per kept
//    track its cluster count (16 bits);
//  * ten byte planes (sector, row, y lo/hi, zeta bytes 0-3, count lo/hi),
//    each coded with a static 256-entry table summing to 4096 (floor-scaled
//    counts, at least 1 for a present symbol, the difference to 4096 taken by
//    the largest entries, lower symbol first) in independent chunks of 4096
//    symbols (32-bit state in [2^23, 2^31), byte renormalisation, symbols
//    coded last to first; a chunk is its final state, 4 bytes little endian,
//    then the emitted bytes in decoding order);
//  * blob: u32 magic 'O2CT', version 1, tracks, track clusters, other
//    clusters, streams (10); per stream u32 symbols, u32 chunks, u16 freq[256],
//    u32 chunk bytes[]; then the chunk payloads in stream and chunk order.
//
// Parallel structure: the two ordered lists (first clusters of kept tracks
// over input indices, clusters on no track over sorted hits) come from the
// warp-ballot compaction; symbols are written at positions known from a scan
// of the track lengths; histograms per chunk in shared memory; one thread
// codes one chunk; a scan of the chunk sizes places the payloads.
#include "o2tpc_internal.cuh"
#include "o2tpc_kernels.cuh"

namespace o2tpc {

namespace {

constexpr int kCtfScaleBits = 12;
constexpr unsigned kCtfM = 1u << kCtfScaleBits;
constexpr unsigned kCtfL = 1u << 23;
constexpr int kCtfChunk = 4096;
constexpr int kCtfStreams = 10;
constexpr float kCtfMaxQpt = 10.f;  // 1 / GeV

__device__ inline long long fdiv64(long long a, long long b) {  // floor division, b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

struct Clu {
  int sec, row, y, z;
};

// The symbols of one cluster of the sequence at position pos.
__device__ inline void emit(uint8_t* sym, long long nSeq, long long pos, const Clu& c, const Clu& prev, bool has2,
                            const Clu& c0, const Clu& c1) {
  long long py = prev.y, pz = prev.z;
  if (has2) {
    py = (long long)c1.y + fdiv64((long long)(c1.y - c0.y) * (c.row - c1.row), c1.row - c0.row);
    pz = (long long)c1.z + fdiv64((long long)(c1.z - c0.z) * (c.row - c1.row), c1.row - c0.row);
  }
  const short ry = (short)(unsigned short)(unsigned long long)((long long)c.y - py);
  const int rz = (int)(unsigned)(unsigned long long)((long long)c.z - pz);
  const unsigned short zy = (unsigned short)(((unsigned short)ry << 1) ^ (unsigned short)(ry >> 15));
  const unsigned zz = ((unsigned)rz << 1) ^ (unsigned)(rz >> 31);
  sym[pos] = (uint8_t)(((c.sec - prev.sec) % 36 + 36) % 36);
  sym[nSeq + pos] = (uint8_t)((c.row - prev.row) & 0xff);
  sym[2 * nSeq + pos] = (uint8_t)zy;
  sym[3 * nSeq + pos] = (uint8_t)(zy >> 8);
  sym[4 * nSeq + pos] = (uint8_t)zz;
  sym[5 * nSeq + pos] = (uint8_t)(zz >> 8);
  sym[6 * nSeq + pos] = (uint8_t)(zz >> 16);
  sym[7 * nSeq + pos] = (uint8_t)(zz >> 24);
}

__device__ inline int find_row_of(const RowGrid* __restrict__ grid, int nRows, int h) {
  int lo = 0, hi = nRows;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (grid[m].start <= h) lo = m + 1;
    else hi = m;
  }
  return lo - 1;
}

__device__ inline Clu sorted_clu(const RowGrid* __restrict__ grid, int nRows, const int2* __restrict__ syz, int s) {
  const int R = find_row_of(grid, nRows, s);
  const int rr = R % kRowsPerTF;
  const int2 p = syz[s];
  return Clu{rr / kNRow, rr % kNRow, p.x, p.y};
}

// Last cluster of the chain of track t.
__device__ inline Clu track_last(int t, const int* __restrict__ heads, const SectorTrackBufs& sb,
                                 const int* __restrict__ next) {
  int c = heads[t];
  for (int j = 1, d = next[c]; d >= 0 && j < kMaxChain; d = next[d], ++j) c = d;
  const int h = sb.off[c + 1] - 1;
  const int2 p = sb.yz[h];
  return Clu{sb.sector[c], sb.rows[h], p.x, p.y};
}

}  // namespace

// Marks the input clusters of every track and the first cluster of every
// kept track (flag, and the track at that index).
__global__ void k_ctf_mark(const int* __restrict__ nTrkDev, OutBufs ob, const TFDesc* __restrict__ tfs,
                           uint8_t* __restrict__ onTrack, int* __restrict__ firstFlag, int* __restrict__ trkAtFirst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nTrkDev) return;
  const int tf = ob.endsR[t].y;
  const int base = tfs[tf].inBase;
  const int a = ob.off[t], b = ob.off[t + 1];
  for (int i = a; i < b; ++i) onTrack[base + ob.cl[i]] = 1;
  const float q = ob.par[(size_t)t * 5 + 4];
  if (b > a && q >= -kCtfMaxQpt && q <= kCtfMaxQpt) {
    firstFlag[base + ob.cl[a]] = 1;
    trkAtFirst[base + ob.cl[a]] = t;
  }
}

__global__ void k_ctf_unflag(const int* __restrict__ nDev, const int* __restrict__ sorig,
                             const uint8_t* __restrict__ onTrack, int* __restrict__ unFlag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *nDev) return;
  unFlag[s] = onTrack[sorig[s]] ? 0 : 1;
}

__global__ void k_ctf_canon(const int* __restrict__ nKeptDev, const int* __restrict__ canonFirst,
                            const int* __restrict__ trkAtFirst, OutBufs ob, int* __restrict__ canonTrk,
                            int* __restrict__ len) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nKeptDev) return;
  const int t = trkAtFirst[canonFirst[k]];
  canonTrk[k] = t;
  len[k] = ob.off[t + 1] - ob.off[t];
}

__global__ void k_ctf_inbase(int nTF, const TFDesc* __restrict__ tfs, const int* __restrict__ nDev,
                             int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > nTF) return;
  out[i] = (i == nTF) ? *nDev : tfs[i].inBase;
}

// Per (TF, stream): first symbol, symbol count, first chunk, chunk count;
// the total chunk count in *nChunks.  One thread (a few hundred entries).
__global__ void k_ctf_streams(int nTF, const int* __restrict__ tfKt, const int* __restrict__ tfUn,
                              const int* __restrict__ lenScan, long long nSeqCap, long long nTrkCap,
                              CtfStream* __restrict__ sd, int* __restrict__ nChunks, int* __restrict__ tfCounts) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int chunk = 0;
  for (int tf = 0; tf < nTF; ++tf) {
    const int k0 = tfKt[tf], k1 = tfKt[tf + 1];
    const int u0 = tfUn[tf], u1 = tfUn[tf + 1];
    const long long seqBase = (long long)lenScan[k0] + u0;
    const long long nTc = (long long)lenScan[k1] - lenScan[k0];
    const long long nSeq = nTc + (u1 - u0);
    tfCounts[tf * 3] = k1 - k0;
    tfCounts[tf * 3 + 1] = (int)nTc;
    tfCounts[tf * 3 + 2] = u1 - u0;
    for (int s = 0; s < kCtfStreams; ++s) {
      CtfStream& d = sd[tf * kCtfStreams + s];
      if (s < 8) {
        d.start = (long long)s * nSeqCap + seqBase;
        d.count = nSeq;
      } else {
        d.start = 8 * nSeqCap + (long long)(s - 8) * nTrkCap + k0;
        d.count = k1 - k0;
      }
      d.chunk0 = chunk;
      d.nChunks = (int)((d.count + kCtfChunk - 1) / kCtfChunk);
      chunk += d.nChunks;
    }
  }
  *nChunks = chunk;
}

// Symbols of the kept tracks' clusters: one warp per track walks its chain,
// 32 consecutive clusters of a segment at a time (coalesced loads and byte
// stores).  Within a sector segment the rows ascend, and neighbouring
// segments of a chain lie in different sectors, so a cluster has the two
// same-segment predecessors of the track model exactly when it is at least
// the third of its segment.
__global__ void __launch_bounds__(128) k_ctf_emit_tracks(const int* __restrict__ nKeptDev,
                                                         const int* __restrict__ canonTrk,
                                                         const int* __restrict__ lenScan,
                                                         const int* __restrict__ tfKt, const int* __restrict__ tfUn,
                                                         OutBufs ob, const int* __restrict__ heads, SectorTrackBufs sb,
                                                         MergeBufs mb, long long nSeq, uint8_t* __restrict__ sym) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (k >= *nKeptDev) return;  // uniform over the warp
  const int t = canonTrk[k];
  const int tf = ob.endsR[t].y;
  Clu prev{0, 0, 0, 0};  // previous cluster of the sequence
  if (k > tfKt[tf]) prev = track_last(canonTrk[k - 1], heads, sb, mb.next);
  long long pos = (long long)lenScan[k] + tfUn[tf];
  int c = heads[t];
  for (int j = 0; c >= 0 && j < kMaxChain; c = mb.next[c], ++j) {
    const int sec = sb.sector[c];
    const int a = sb.off[c], b = sb.off[c + 1];
    Clu l1 = prev, l2 = prev;  // the two clusters before the current group
    for (int g = a; g < b; g += 32) {
      const int i = g + lane;
      const bool valid = i < b;
      const int2 p = valid ? sb.yz[i] : make_int2(0, 0);
      const int rw = valid ? (int)sb.rows[i] : 0;
      const Clu cu{sec, rw, p.x, p.y};
      // cluster i - 1 and i - 2 of the sequence
      Clu m1, m2;
      m1.sec = sec;
      m1.y = __shfl_up_sync(full, cu.y, 1);
      m1.z = __shfl_up_sync(full, cu.z, 1);
      m1.row = __shfl_up_sync(full, cu.row, 1);
      m2.sec = sec;
      m2.y = __shfl_up_sync(full, cu.y, 2);
      m2.z = __shfl_up_sync(full, cu.z, 2);
      m2.row = __shfl_up_sync(full, cu.row, 2);
      if (lane == 0) {
        m1 = l1;
        m2 = l2;
      } else if (lane == 1) {
        m2 = l1;
      }
      const int qs = i - a;  // index inside the segment
      if (valid) emit(sym, nSeq, pos + qs, cu, m1, qs >= 2, m2, m1);
      // carry the last two clusters of the group
      const int nv = min(32, b - g);
      Clu n1, n2;
      n1.sec = sec;
      n1.y = __shfl_sync(full, cu.y, nv - 1);
      n1.z = __shfl_sync(full, cu.z, nv - 1);
      n1.row = __shfl_sync(full, cu.row, nv - 1);
      n2.sec = sec;
      n2.y = __shfl_sync(full, cu.y, max(nv - 2, 0));
      n2.z = __shfl_sync(full, cu.z, max(nv - 2, 0));
      n2.row = __shfl_sync(full, cu.row, max(nv - 2, 0));
      if (nv < 2) n2 = l1;
      l2 = n2;
      l1 = n1;
    }
    prev = l1;
    pos += b - a;
  }
}

// Symbols of the clusters on no track (sorted-hit order).
__global__ void k_ctf_emit_free(const int* __restrict__ nUnDev, const int* __restrict__ unList,
                                const RowGrid* __restrict__ grid, int nRows, const int2* __restrict__ syz,
                                const int* __restrict__ lenScan, const int* __restrict__ tfKt,
                                const int* __restrict__ tfUn, const int* __restrict__ canonTrk,
                                const int* __restrict__ heads, SectorTrackBufs sb, MergeBufs mb, long long nSeq,
                                uint8_t* __restrict__ sym) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= *nUnDev) return;
  const int s = unList[j];
  const Clu cu = sorted_clu(grid, nRows, syz, s);
  const int tf = find_row_of(grid, nRows, s) / kRowsPerTF;
  Clu prev{0, 0, 0, 0};
  if (j > tfUn[tf]) prev = sorted_clu(grid, nRows, syz, unList[j - 1]);
  else if (tfKt[tf + 1] > tfKt[tf]) prev = track_last(canonTrk[tfKt[tf + 1] - 1], heads, sb, mb.next);
  const long long pos = (long long)lenScan[tfKt[tf + 1]] + j;
  emit(sym, nSeq, pos, cu, prev, false, cu, cu);
}

__global__ void k_ctf_emit_len(const int* __restrict__ nKeptDev, const int* __restrict__ len, long long nSeqCap,
                               long long nTrkCap, uint8_t* __restrict__ sym) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nKeptDev) return;
  sym[8 * nSeqCap + k] = (uint8_t)len[k];
  sym[8 * nSeqCap + nTrkCap + k] = (uint8_t)(len[k] >> 8);
}

// Stream of chunk c (the first stream whose chunk range ends after c).
__device__ inline int stream_of_chunk(const CtfStream* __restrict__ sd, int nSd, int c) {
  int lo = 0, hi = nSd;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (sd[m].chunk0 + sd[m].nChunks <= c) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// One block per kCtfHistChunks consecutive chunks (mostly one stream): a
// shared-memory histogram, flushed to the stream's global one whenever the
// stream changes.
constexpr int kCtfHistChunks = 32;
__global__ void __launch_bounds__(256) k_ctf_hist(const int* __restrict__ nChunksDev, const CtfStream* __restrict__ sd,
                                                  int nSd, const uint8_t* __restrict__ sym,
                                                  unsigned* __restrict__ hist) {
  __shared__ unsigned h[256];
  const int nCh = *nChunksDev;
  const int c0 = blockIdx.x * kCtfHistChunks;
  if (c0 >= nCh) return;
  const int c1 = min(nCh, c0 + kCtfHistChunks);
  int s = stream_of_chunk(sd, nSd, c0);
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int c = c0; c < c1;) {
    while (sd[s].chunk0 + sd[s].nChunks <= c) ++s;
    const CtfStream d = sd[s];
    const int ce = min(c1, d.chunk0 + d.nChunks);  // this stream's part of the range
    const long long a = (long long)(c - d.chunk0) * kCtfChunk;
    const long long e = min(d.count, (long long)(ce - d.chunk0) * kCtfChunk);
    const uint8_t* p = sym + d.start;
    // runs of equal symbols seen by a thread are added at once (most byte
    // planes are dominated by one symbol)
    unsigned cur = 256u, run = 0;
    for (long long i = a + threadIdx.x; i < e; i += blockDim.x) {
      const unsigned v = p[i];
      if (v == cur) {
        ++run;
      } else {
        if (run) atomicAdd(&h[cur], run);
        cur = v;
        run = 1;
      }
    }
    if (run) atomicAdd(&h[cur], run);
    __syncthreads();
    if (h[threadIdx.x]) {
      atomicAdd(&hist[s * 256 + threadIdx.x], h[threadIdx.x]);
      h[threadIdx.x] = 0;
    }
    __syncthreads();
    c = ce;
  }
}

// One thread per (TF, stream): the normalised table and its cumulative sums.
__global__ void k_ctf_norm(int nSd, const unsigned* __restrict__ hist, uint16_t* __restrict__ freq,
                           uint2* __restrict__ enc, int* __restrict__ degen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nSd) return;
  const unsigned* c = hist + s * 256;
  uint16_t* f = freq + s * 256;
  unsigned long long n = 0;
  for (int k = 0; k < 256; ++k) n += c[k];
  long long sum = 0;
  for (int k = 0; k < 256; ++k) {
    unsigned long long v = 0;
    if (c[k]) {
      v = (unsigned long long)c[k] * kCtfM / n;
      if (v < 1) v = 1;
    }
    f[k] = (uint16_t)v;
    sum += (long long)v;
  }
  long long dlt = n ? (long long)kCtfM - sum : 0;
  while (dlt != 0) {
    int best = -1;
    for (int k = 0; k < 256; ++k)
      if (f[k] && (best < 0 || f[k] > f[best])) best = k;
    if (dlt > 0) {
      f[best] = (uint16_t)(f[best] + dlt);
      dlt = 0;
    } else {
      long long take = (long long)f[best] - 1;
      if (take > -dlt) take = -dlt;
      f[best] = (uint16_t)(f[best] - take);
      dlt += take;
    }
  }
  // coding entries: cumulative start | frequency << 16, and 1 / frequency
  unsigned acc = 0;
  int dg = 0;
  for (int k = 0; k < 256; ++k) {
    enc[s * 256 + k] = make_uint2(acc | ((unsigned)f[k] << 16), __float_as_uint(f[k] ? 1.0f / (float)f[k] : 0.f));
    acc += f[k];
    dg |= f[k] == kCtfM;
  }
  degen[s] = dg;
}

// One thread per chunk: rANS from the last symbol to the first; the emitted
// bytes go backwards from the end of the chunk's scratch slot (gathered into
// 32-bit words), the final state in front of them.  bytes[c] = 4 + emitted.
// A table with one symbol of frequency 4096 codes nothing: the state stays
// at its initial value.
__global__ void __launch_bounds__(128) k_ctf_encode(const int* __restrict__ nChunksDev, const CtfStream* __restrict__ sd,
                                                    int nSd, const uint8_t* __restrict__ sym,
                                                    const uint2* __restrict__ enc, const int* __restrict__ degen,
                                                    uint8_t* __restrict__ scratch, int* __restrict__ bytes) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= *nChunksDev) return;
  const int s = stream_of_chunk(sd, nSd, c);
  const CtfStream d = sd[s];
  const long long a = (long long)(c - d.chunk0) * kCtfChunk;
  const int n = (int)min((long long)kCtfChunk, d.count - a);
  uint8_t* out = scratch + (size_t)c * kCtfChunkBytes;
  unsigned x = kCtfL;
  int q = kCtfChunkBytes;  // emitted bytes fill [q, kCtfChunkBytes)
  if (!degen[s]) {
    const uint8_t* p = sym + d.start + a;
    const uint2* tab = enc + s * 256;
    unsigned w = 0;  // bytes not yet stored, the latest emitted in the low byte
    int nw = 0;
    for (int i = n - 1; i >= 0; --i) {
      const uint2 e = tab[p[i]];
      const unsigned fs = e.x >> 16, cs = e.x & 0xffffu;
      const unsigned xmax = ((kCtfL >> kCtfScaleBits) << 8) * fs;
      while (x >= xmax) {
        w = (w << 8) | (x & 0xffu);
        x >>= 8;
        if (++nw == 4) {
          q -= 4;
          *reinterpret_cast<unsigned*>(out + q) = w;
          nw = 0;
        }
      }
      // x / fs: here x < 2^19 fs, so the quotient is below 2^19 and the
      // single-precision estimate (relative error < 2^-22) is off by at most
      // one, which one remainder test corrects
      unsigned qt = __float2uint_rz(__uint2float_rn(x) * __uint_as_float(e.y));
      int r = (int)(x - qt * fs);
      if (r < 0) {
        --qt;
        r += (int)fs;
      } else if (r >= (int)fs) {
        ++qt;
        r -= (int)fs;
      }
      x = (qt << kCtfScaleBits) + (unsigned)r + cs;
    }
    for (int k = 0; k < nw; ++k) out[--q] = (uint8_t)(w >> (8 * (nw - 1 - k)));
  }
  out[q - 4] = (uint8_t)x;
  out[q - 3] = (uint8_t)(x >> 8);
  out[q - 2] = (uint8_t)(x >> 16);
  out[q - 1] = (uint8_t)(x >> 24);
  bytes[c] = kCtfChunkBytes - q + 4;
}

// Per TF: header size and payload size, then the TF blobs' offsets (one
// thread; tfBlob[nTF] is the total).
__global__ void k_ctf_layout(int nTF, const CtfStream* __restrict__ sd, const int* __restrict__ payOff,
                             long long* __restrict__ tfBlob, long long* __restrict__ tfHead) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  long long o = 0;
  for (int tf = 0; tf < nTF; ++tf) {
    long long h = 24;
    for (int s = 0; s < kCtfStreams; ++s) h += 8 + 512 + 4ll * sd[tf * kCtfStreams + s].nChunks;
    const CtfStream& first = sd[tf * kCtfStreams];
    const CtfStream& last = sd[tf * kCtfStreams + kCtfStreams - 1];
    const long long pay = (long long)payOff[last.chunk0 + last.nChunks] - payOff[first.chunk0];
    tfBlob[tf] = o;
    tfHead[tf] = h;
    o += h + pay;
  }
  tfBlob[nTF] = o;
}

__device__ inline void put32(uint8_t* p, unsigned v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}

// One block per TF: the header (counts, tables, chunk sizes).
__global__ void k_ctf_header(int nTF, const CtfStream* __restrict__ sd, const int* __restrict__ tfCounts,
                             const uint16_t* __restrict__ freq, const int* __restrict__ bytes,
                             const long long* __restrict__ tfBlob, uint8_t* __restrict__ blob) {
  const int tf = blockIdx.x;
  if (tf >= nTF) return;
  uint8_t* b = blob + tfBlob[tf];
  if (threadIdx.x == 0) {
    put32(b, 0x5443324Fu);
    put32(b + 4, 1);
    put32(b + 8, (unsigned)tfCounts[tf * 3]);
    put32(b + 12, (unsigned)tfCounts[tf * 3 + 1]);
    put32(b + 16, (unsigned)tfCounts[tf * 3 + 2]);
    put32(b + 20, kCtfStreams);
  }
  long long o = 24;
  for (int s = 0; s < kCtfStreams; ++s) {
    const int id = tf * kCtfStreams + s;
    const CtfStream d = sd[id];
    uint8_t* h = b + o;
    if (threadIdx.x == 0) {
      put32(h, (unsigned)d.count);
      put32(h + 4, (unsigned)d.nChunks);
    }
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
      const uint16_t v = freq[id * 256 + k];
      h[8 + 2 * k] = (uint8_t)v;
      h[9 + 2 * k] = (uint8_t)(v >> 8);
    }
    o += 8 + 512 + 4ll * d.nChunks;  // the chunk sizes are written by k_ctf_copy
  }
}

// One block per chunk: its size into the stream's header, its payload from
// the scratch slot into the blob.
__global__ void k_ctf_copy(const int* __restrict__ nChunksDev, int nTF, const CtfStream* __restrict__ sd,
                           const int* __restrict__ bytes, const int* __restrict__ payOff,
                           const long long* __restrict__ tfBlob, const long long* __restrict__ tfHead,
                           const uint8_t* __restrict__ scratch, uint8_t* __restrict__ blob) {
  const int c = blockIdx.x;
  if (c >= *nChunksDev) return;
  int tf = 0;
  {
    int lo = 0, hi = nTF;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      const CtfStream& last = sd[m * kCtfStreams + kCtfStreams - 1];
      if (last.chunk0 + last.nChunks <= c) lo = m + 1;
      else hi = m;
    }
    tf = lo;
  }
  const int first = sd[tf * kCtfStreams].chunk0;
  uint8_t* dst = blob + tfBlob[tf] + tfHead[tf] + (payOff[c] - payOff[first]);
  const int nb = bytes[c];
  if (threadIdx.x == 0) {
    const int s = stream_of_chunk(sd, nTF * kCtfStreams, c);
    long long h = 24;
    for (int k = tf * kCtfStreams; k < s; ++k) h += 8 + 512 + 4ll * sd[k].nChunks;
    put32(blob + tfBlob[tf] + h + 520 + 4ll * (c - sd[s].chunk0), (unsigned)nb);
  }
  const uint8_t* src = scratch + (size_t)c * kCtfChunkBytes + (kCtfChunkBytes - nb);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------------------- launchers
int ctf_chunk_cap(long long nSeqCap, long long nTrkCap, int nTF) {
  return (int)(8 * (nSeqCap / kCtfChunk + nTF + 1) + 2 * (nTrkCap / kCtfChunk + nTF + 1));
}

void launch_ctf_symbols(int n, const int* nDev, int nTrk, const int* nTrkDev, int nTF, const TFDesc* tfs,
                        const RowGrid* grid, int nRows, const int2* syz, const int* sorig, const int* heads,
                        SectorTrackBufs sb, MergeBufs mb, OutBufs ob, CtfBufs cb, int* tileCnt, int* tileOff,
                        int* overflow, int* scratch, cudaStream_t st) {
  cudaMemsetAsync(cb.onTrack, 0, (size_t)n + 1, st);
  cudaMemsetAsync(cb.firstFlag, 0, sizeof(int) * ((size_t)n + 1), st);
  if (nTrk > 0) {
    k_ctf_mark<<<(nTrk + 255) / 256, 256, 0, st>>>(nTrkDev, ob, tfs, cb.onTrack, cb.firstFlag, cb.trkAtFirst);
    ++g_launch_count;
  }
  // kept tracks by first input index; clusters on no track in sorted order
  launch_ballot_count(n, nDev, cb.firstFlag, tileCnt, tileOff, cb.counts, nTrk, overflow, scratch, st);
  launch_ballot_compact(n, nDev, cb.firstFlag, tileOff, cb.canonFirst, nTrk, overflow, st);
  if (n > 0) {
    k_ctf_unflag<<<(n + 255) / 256, 256, 0, st>>>(nDev, sorig, cb.onTrack, cb.unFlag);
    ++g_launch_count;
  }
  launch_ballot_count(n, nDev, cb.unFlag, tileCnt, tileOff, cb.counts + 1, n, overflow, scratch, st);
  launch_ballot_compact(n, nDev, cb.unFlag, tileOff, cb.unList, n, overflow, st);
  if (nTrk > 0) {
    k_ctf_canon<<<(nTrk + 255) / 256, 256, 0, st>>>(cb.counts, cb.canonFirst, cb.trkAtFirst, ob, cb.canonTrk,
                                                      cb.len);
    ++g_launch_count;
  }
  scan_exclusive(cb.len, cb.lenScan, nTrk, cb.counts, scratch, st);
  k_ctf_inbase<<<(nTF + 1 + 63) / 64, 64, 0, st>>>(nTF, tfs, nDev, cb.inBase);
  ++g_launch_count;
  launch_lower_bounds(cb.canonFirst, cb.counts, cb.inBase, nTF + 1, cb.tfKt, st);
  launch_tf_ranges(nTF, grid, cb.unList, cb.counts + 1, cb.tfUn, st);
  k_ctf_streams<<<1, 1, 0, st>>>(nTF, cb.tfKt, cb.tfUn, cb.lenScan, cb.nSeqCap, cb.nTrkCap, cb.sd, cb.counts + 2,
                                 cb.tfCounts);
  ++g_launch_count;
  if (nTrk > 0) {
    k_ctf_emit_tracks<<<(int)(((long long)nTrk * 32 + 127) / 128), 128, 0, st>>>(
        cb.counts, cb.canonTrk, cb.lenScan, cb.tfKt, cb.tfUn, ob, heads, sb, mb, cb.nSeqCap, cb.sym);
    k_ctf_emit_len<<<(nTrk + 255) / 256, 256, 0, st>>>(cb.counts, cb.len, cb.nSeqCap, cb.nTrkCap, cb.sym);
    g_launch_count += 2;
  }
  if (n > 0) {
    k_ctf_emit_free<<<(n + 255) / 256, 256, 0, st>>>(cb.counts + 1, cb.unList, grid, nRows, syz, cb.lenScan, cb.tfKt,
                                                       cb.tfUn, cb.canonTrk, heads, sb, mb, cb.nSeqCap, cb.sym);
    ++g_launch_count;
  }
  const int nSd = nTF * kCtfStreams;
  cudaMemsetAsync(cb.hist, 0, sizeof(unsigned) * 256 * nSd, st);
  k_ctf_hist<<<(cb.chunkCap + kCtfHistChunks - 1) / kCtfHistChunks, 256, 0, st>>>(cb.counts + 2, cb.sd, nSd, cb.sym,
                                                                                  cb.hist);
  k_ctf_norm<<<(nSd + 63) / 64, 64, 0, st>>>(nSd, cb.hist, cb.freq, cb.enc, cb.degen);
  k_ctf_encode<<<(cb.chunkCap + 127) / 128, 128, 0, st>>>(cb.counts + 2, cb.sd, nSd, cb.sym, cb.enc, cb.degen,
                                                          cb.scratch, cb.bytes);
  g_launch_count += 3;
  scan_exclusive(cb.bytes, cb.payOff, cb.chunkCap, cb.counts + 2, scratch, st);
  k_ctf_layout<<<1, 1, 0, st>>>(nTF, cb.sd, cb.payOff, cb.tfBlob, cb.tfHead);
  ++g_launch_count;
}

void launch_ctf_blob(int nTF, CtfBufs cb, uint8_t* blob, cudaStream_t st) {
  k_ctf_header<<<nTF, 256, 0, st>>>(nTF, cb.sd, cb.tfCounts, cb.freq, cb.bytes, cb.tfBlob, blob);
  k_ctf_copy<<<cb.chunkCap, 256, 0, st>>>(cb.counts + 2, nTF, cb.sd, cb.bytes, cb.payOff, cb.tfBlob, cb.tfHead,
                                          cb.scratch, blob);
  g_launch_count += 2;
}

}  // namespace o2tpc
