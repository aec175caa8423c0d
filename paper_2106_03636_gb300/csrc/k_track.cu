// k_track.cu - TrackletConstructor, TrackletSelector and the sector-track fits.
//
// A tracklet starts at a chain head: the chain's hits are fitted with the
// FP32 Kalman filter, the track is followed outward row by row (best hit in a
// +-3 sigma window, chi2 <= 18, stop after 4 rows without a hit or at
// |sin phi| > 0.95), then refitted inward from its top hit and followed below
// the chain start.  The selector gives every hit to the longest tracklet
// holding it (ties: the earlier start) through a 64-bit atomicMax of
// (nHits << 32 | ~id), which makes the result independent of thread order,
// splits tracklets at gaps of more than 4 rows and keeps segments of >= 10
// owned hits as sector tracks, each refitted outward and inward.
#include <algorithm>

#include "o2tpc_kernels.cuh"

namespace o2tpc {

// Hit coordinates in cm relative to per-fit origins (yref, zref in integer
// units): the fits then work on small magnitudes, where single precision keeps
// its digits.
__device__ inline float hit_y(int yu, int yref) { return (float)(yu - yref) * 0.00625f; }
__device__ inline float hit_z(int zu, int zref, float zunit) { return (float)(zu - zref) * zunit; }

// Row (batch-global) holding sorted hit h.
__device__ inline int find_row(const RowGrid* __restrict__ grid, int nRows, int h) {
  int lo = 0, hi = nRows;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (grid[m].start <= h) lo = m + 1;
    else hi = m;
  }
  return lo - 1;
}

__device__ inline int clamp_i(float v) { return (int)fminf(fmaxf(v, -1.0e9f), 1.0e9f); }

// Best hit of a row inside the +-3 sigma window of the prediction (ties: the
// smaller sorted index); -1 if none has chi2 <= kChi2Follow.  The best hit's
// coordinates come back in *pbest.
__device__ int search_row(const RowGrid& g, int npads, const int* __restrict__ cellStart,
                          const int2* __restrict__ syz, const KState<float>& s, int yref, int zref,
                          float zunit, float izunit, int2* pbest) {
  if (g.count == 0) return -1;
  const float sy2 = s.C[0] + kSigY * kSigY, sz2 = s.C[2] + kSigZ * kSigZ;
  const float wy = 3.f * sqrtf(sy2), wz = 3.f * sqrtf(sz2);
  if (!(wy < 1e4f) || !(wz < 1e4f) || !isfinite(s.p[0]) || !isfinite(s.p[1])) return -1;
  // the cell rectangle only has to cover the window: one unit of slack on
  // each side absorbs the rounding of the float products
  const int ylo = yref + clamp_i(floorf((s.p[0] - wy) * 160.f)) - 1;
  const int yhi = yref + clamp_i(ceilf((s.p[0] + wy) * 160.f)) + 1;
  const int zlo = zref + clamp_i(floorf((s.p[1] - wz) * izunit)) - 1;
  const int zhi = zref + clamp_i(ceilf((s.p[1] + wz) * izunit)) + 1;
  int iy0, iy1, iz0, iz1;
  if (!cell_range(g, npads, ylo, yhi, zlo, zhi, iy0, iy1, iz0, iz1)) return -1;
  const float isy2 = 1.f / sy2, isz2 = 1.f / sz2;
  int best = -1;
  float bchi = 0.f;
  int2 bp = make_int2(0, 0);
  for (int iz = iz0; iz <= iz1; ++iz) {
    const int a = __ldg(cellStart + g.cellBase + iz * g.ny + iy0);
    const int b = __ldg(cellStart + g.cellBase + iz * g.ny + iy1 + 1);
    for (int h = a; h < b; ++h) {
      const int2 p = __ldg(syz + h);
      const float dy = hit_y(p.x, yref) - s.p[0], dz = hit_z(p.y, zref, zunit) - s.p[1];
      if (fabsf(dy) > wy || fabsf(dz) > wz) continue;
      const float chi = dy * dy * isy2 + dz * dz * isz2;
      if (chi > kChi2Follow) continue;
      if (best < 0 || chi < bchi || (chi == bchi && h < best)) {
        best = h;
        bchi = chi;
        bp = p;
      }
    }
  }
  *pbest = bp;
  return best;
}

__device__ inline void reset_cov(KState<float>& s) {
#pragma unroll
  for (int i = 0; i < 15; ++i) s.C[i] = 0.f;
  s.C[0] = kSigY * kSigY;
  s.C[2] = kSigZ * kSigZ;
  s.C[5] = 0.04f;
  s.C[9] = 0.25f;
  s.C[14] = 400.f;
}

// Stores a state with y back in absolute cm (yref in units).
__device__ inline void store_state(float* dst, const KState<float>& s, int yref) {
  dst[0] = s.x;
#pragma unroll
  for (int i = 0; i < 5; ++i) dst[1 + i] = s.p[i];
  dst[1] = s.p[0] + (float)yref * 0.00625f;
#pragma unroll
  for (int i = 0; i < 15; ++i) dst[6 + i] = s.C[i];
}
// Stores a state as it is (y relative to the fit's origin): the hand-over
// between the passes of the tracklet constructor.
__device__ inline void store_raw(float* dst, const KState<float>& s) {
  dst[0] = s.x;
#pragma unroll
  for (int i = 0; i < 5; ++i) dst[1 + i] = s.p[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) dst[6 + i] = s.C[i];
}
__device__ inline void load_state(KState<float>& s, const float* src) {
  s.x = src[0];
#pragma unroll
  for (int i = 0; i < 5; ++i) s.p[i] = src[1 + i];
#pragma unroll
  for (int i = 0; i < 15; ++i) s.C[i] = src[6 + i];
}

// K7: the TrackletConstructor in four passes, one persistent kernel each:
// (a) chain fit, (b) outward following, (c) inward refit of the attached
// hits, (d) inward following below the chain start.  Within a pass every
// lane runs the same loop body (transport, then either the next known hit or
// a row search, then the update), so a warp stays converged; lanes take the
// next tracklet from a global counter as soon as theirs is done.  Between the
// passes a tracklet's state waits in tb.state (21 floats), its hit count in
// tb.nasc and its row base in tb.rbase; tb.nhits is written by the last pass
// (0: dropped).  Results do not depend on which thread builds which tracklet.

// (a) chain fit: seed from the first and third chain hits, then one update
// per chain hit.  A transport failure drops the tracklet.
__global__ void __launch_bounds__(128) k_tl_chain(const int* __restrict__ nTlDev, int* __restrict__ counter, const int* __restrict__ starts,
                                                  const int* __restrict__ up, const RowGrid* __restrict__ grid,
                                                  int nRows, const int2* __restrict__ syz,
                                                  const GeomConst* __restrict__ G, TrackletBufs tb) {
  const float zunit = G->zunit, bzc = G->bzc;
  const int nTl = *nTlDev;
  for (;;) {
    const int k = atomicAdd(counter, 1);
    if (k >= nTl) return;
    const int h0 = starts[k];
    const int R0 = find_row(grid, nRows, h0);
    const int r0 = (R0 % kRowsPerTF) % kNRow;
    int* H = tb.hits + (size_t)k * kMaxTlHits;
    uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    const int2 a0 = syz[h0];
    const int zref = a0.y, yref = a0.x;
    tb.zref[k] = zref;
    tb.rbase[k] = R0 - r0;
    const int h1 = up[h0];
    const int2 a2 = syz[up[h1]];
    const float x0 = G->rowx[r0], x2 = G->rowx[r0 + 2];
    const float dx = x2 - x0, dy = hit_y(a2.x, yref) - hit_y(a0.x, yref);
    const float tphi = dy / dx;
    const float s0 = tphi / sqrtf(1.f + tphi * tphi);
    const float t0 = (hit_z(a2.y, zref, zunit) - hit_z(a0.y, zref, zunit)) / sqrtf(dx * dx + dy * dy);
    KState<float> st;
    kf_reset<float>(st, x0, hit_y(a0.x, yref), hit_z(a0.y, zref, zunit), s0, t0, 0.f);
    H[0] = h0;
    Rw[0] = (uint8_t)r0;
    int nc = 1, hit = h1;
    bool dropped = false;
    while (hit >= 0 && nc < kNRow - r0) {
      const int row = r0 + nc;
      const int2 hp = syz[hit];  // both loads in flight during the transport
      const int next = up[hit];
      if (kf_prop<float>(st, G->rowx[row], bzc) != 0) {
        dropped = true;
        break;
      }
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr);
      H[nc] = hit;
      Rw[nc] = (uint8_t)row;
      ++nc;
      hit = next;
    }
    tb.nasc[k] = dropped ? 0 : nc;
    if (dropped) tb.nhits[k] = 0;
    else store_raw(tb.state + (size_t)k * 21, st);
  }
}

// Following (passes b and d): from row r in steps of dir, transport, search
// the +-3 sigma window, update with the best hit; stop after kMaxMiss rows
// without a hit, at the row range end, on a transport failure or when
// |sin phi| > kSinFollow.  The state after the last accepted hit is kept in
// shared memory (one column per thread) and returned in st.  Appends the
// hits at H[n..]; returns the new count.
template <int kDir>
__device__ inline int follow(KState<float>& st, float (*s_last)[128], int r, int n, int* H, uint8_t* Rw, int* top,
                             int Rs, int yref, int zref, const RowGrid* __restrict__ grid,
                             const int* __restrict__ cellStart, const int2* __restrict__ syz,
                             const GeomConst* __restrict__ G, float zunit, float izunit, float bzc) {
  auto save_last = [&](const KState<float>& q) {
    s_last[0][threadIdx.x] = q.x;
#pragma unroll
    for (int j = 0; j < 5; ++j) s_last[1 + j][threadIdx.x] = q.p[j];
#pragma unroll
    for (int j = 0; j < 15; ++j) s_last[6 + j][threadIdx.x] = q.C[j];
  };
  save_last(st);
  int misses = 0;
  for (; kDir > 0 ? r < kNRow : r >= 0; r += kDir) {
    if (kf_prop<float>(st, G->rowx[r], bzc) != 0 || fabsf(st.p[2]) > kSinFollow) break;
    int2 hp;
    const int hit = search_row(grid[Rs + r], G->npads[r], cellStart, syz, st, yref, zref, zunit, izunit, &hp);
    if (hit >= 0) {
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr);
      H[n] = hit;
      Rw[n] = (uint8_t)r;
      ++n;
      *top = hit;
      save_last(st);
      misses = 0;
    } else if (++misses >= kMaxMiss) {
      break;
    }
  }
  st.x = s_last[0][threadIdx.x];
#pragma unroll
  for (int j = 0; j < 5; ++j) st.p[j] = s_last[1 + j][threadIdx.x];
#pragma unroll
  for (int j = 0; j < 15; ++j) st.C[j] = s_last[6 + j][threadIdx.x];
  return n;
}

// The two following passes are latency bound (dependent grid -> cell -> hit
// loads per row step): they run at 9 CTAs of 128 threads per SM (56
// registers, a few bytes of spill), measured 12 % faster than at 7 CTAs.

// (b) outward following above the chain; then the refit's starting state:
// the last accepted state with the position of the top hit and a fresh
// covariance.
__global__ void __launch_bounds__(128, 9) k_tl_out(const int* __restrict__ nTlDev, int* __restrict__ counter, const RowGrid* __restrict__ grid,
                                                const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                                const GeomConst* __restrict__ G, TrackletBufs tb) {
  __shared__ float s_last[21][128];
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  const int nTl = *nTlDev;
  for (;;) {
    const int k = atomicAdd(counter, 1);
    if (k >= nTl) return;
    const int nc = tb.nasc[k];
    if (nc == 0) continue;
    int* H = tb.hits + (size_t)k * kMaxTlHits;
    uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    const int r0 = Rw[0], Rs = tb.rbase[k], zref = tb.zref[k];
    const int yref = syz[H[0]].x;
    KState<float> st;
    float* S = tb.state + (size_t)k * 21;
    load_state(st, S);
    int top = H[nc - 1];
    const int na = follow<1>(st, s_last, r0 + nc, nc, H, Rw, &top, Rs, yref, zref, grid, cellStart, syz, G, zunit,
                             izunit, bzc);
    const int2 p = syz[top];
    st.p[0] = hit_y(p.x, yref);
    st.p[1] = hit_z(p.y, zref, zunit);
    reset_cov(st);
    tb.nasc[k] = na;
    store_raw(S, st);
  }
}

// (c) inward refit from the top hit through every attached hit; a hit whose
// transport fails is skipped.
__global__ void __launch_bounds__(128) k_tl_refit(const int* __restrict__ nTlDev, int* __restrict__ counter, const int2* __restrict__ syz,
                                                  const GeomConst* __restrict__ G, TrackletBufs tb) {
  const float zunit = G->zunit, bzc = G->bzc;
  const int nTl = *nTlDev;
  for (;;) {
    const int k = atomicAdd(counter, 1);
    if (k >= nTl) return;
    const int na = tb.nasc[k];
    if (na == 0) continue;
    const int* H = tb.hits + (size_t)k * kMaxTlHits;
    const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    const int zref = tb.zref[k];
    const int yref = syz[H[0]].x;
    KState<float> st;
    float* S = tb.state + (size_t)k * 21;
    load_state(st, S);
    for (int i = na - 2; i >= 0; --i) {
      const int2 hp = syz[H[i]];
      if (kf_prop<float>(st, G->rowx[Rw[i]], bzc) != 0) continue;
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr);
    }
    store_raw(S, st);
  }
}

// (d) inward following below the chain start; the state kept is the one at
// the innermost accepted hit.
__global__ void __launch_bounds__(128, 9) k_tl_in(const int* __restrict__ nTlDev, int* __restrict__ counter, const RowGrid* __restrict__ grid,
                                               const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                               const GeomConst* __restrict__ G, TrackletBufs tb) {
  __shared__ float s_last[21][128];
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  const int nTl = *nTlDev;
  for (;;) {
    const int k = atomicAdd(counter, 1);
    if (k >= nTl) return;
    const int na = tb.nasc[k];
    if (na == 0) continue;
    int* H = tb.hits + (size_t)k * kMaxTlHits;
    uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    const int r0 = Rw[0], Rs = tb.rbase[k], zref = tb.zref[k];
    const int yref = syz[H[0]].x;
    KState<float> st;
    float* S = tb.state + (size_t)k * 21;
    load_state(st, S);
    int top = -1;
    const int n = follow<-1>(st, s_last, r0 - 1, na, H, Rw, &top, Rs, yref, zref, grid, cellStart, syz, G, zunit,
                             izunit, bzc);
    tb.nhits[k] = n;
    store_state(S, st, yref);
  }
}


// Ownership keys.  Only tracklets of the same sector can share a hit, so the
// tie-break id is the tracklet's index within its sector (same order as the
// index within the TF): (nHits << 24 | 2^24-1-id) in 32 bits, or the 64-bit
// (nHits << 32 | 2^32-1-id) when a sector holds 2^24 tracklets or more.
__device__ inline unsigned own_key32(int nh, int lid) { return ((unsigned)nh << 24) | (0xFFFFFFu - (unsigned)lid); }
__device__ inline unsigned long long own_key64(int nh, int lid) {
  return ((unsigned long long)(unsigned)nh << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)lid);
}

// First tracklet of every (TF, sector) (start hits are sorted by hit index);
// *wide = 1 when a sector holds 2^24 tracklets or more.
__global__ void k_sector_ranges(int nSec, const RowGrid* __restrict__ grid, const int* __restrict__ starts,
                                const int* __restrict__ nTlDev, int* __restrict__ secBegin, int* __restrict__ wide) {
  const int ts = blockIdx.x * blockDim.x + threadIdx.x;
  if (ts > nSec) return;
  const int nTl = *nTlDev;
  auto lower = [&](int key) {
    int lo = 0, hi = nTl;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (starts[m] < key) lo = m + 1;
      else hi = m;
    }
    return lo;
  };
  const int b = (ts == nSec) ? nTl : lower(grid[ts * kNRow].start);
  secBegin[ts] = b;
  if (ts < nSec) {
    const int e = (ts + 1 == nSec) ? nTl : lower(grid[(ts + 1) * kNRow].start);
    if (e - b >= (1 << 24)) atomicOr(wide, 1);
  }
}

struct OwnCtx {
  const int* secBegin;
  const int* wide;
  void* w;  // unsigned[n] or unsigned long long[n]
};

// Key of tracklet k and whether hit h is owned by it.
struct TlKey {
  bool wide;
  unsigned k32;
  unsigned long long k64;
  __device__ bool owns(const OwnCtx& o, int h) const {
    return wide ? static_cast<const unsigned long long*>(o.w)[h] == k64 : static_cast<const unsigned*>(o.w)[h] == k32;
  }
};
__device__ inline TlKey tl_key(const OwnCtx& o, const TrackletBufs& tb, int k, int nh) {
  const int lid = k - o.secBegin[tb.rbase[k] / kNRow];
  TlKey t;
  t.wide = *o.wide != 0;
  t.k32 = own_key32(nh, lid);
  t.k64 = own_key64(nh, lid);
  return t;
}

// K8a: hit ownership (atomicMax of the key; a hit already holding a larger
// key is skipped without an atomic).
__global__ void k_ownership(const int* __restrict__ nTlDev, OwnCtx o, TrackletBufs tb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nTlDev) return;
  const int nh = tb.nhits[k];
  if (nh < kMinHits) return;
  const TlKey key = tl_key(o, tb, k, nh);
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  if (key.wide) {
    auto* w = static_cast<unsigned long long*>(o.w);
    for (int i = 0; i < nh; ++i) {
      const int h = H[i];
      if (w[h] < key.k64) atomicMax(&w[h], key.k64);
    }
  } else {
    auto* w = static_cast<unsigned*>(o.w);
    for (int i = 0; i < nh; ++i) {
      const int h = H[i];
      if (w[h] < key.k32) atomicMax(&w[h], key.k32);
    }
  }
}

// K8b: segments per tracklet (count pass): owned hits in row order, split at
// gaps of more than kMaxMiss rows, segments of >= kMinHits kept.
__global__ void __launch_bounds__(128) k_segments_count(const int* __restrict__ nTlDev, OwnCtx o, TrackletBufs tb,
                                                        int* __restrict__ nSeg, int* __restrict__ nSegHits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nTlDev) return;
  const int nh = tb.nhits[k];
  int cs = 0, ch = 0;
  if (nh >= kMinHits) {
    const TlKey key = tl_key(o, tb, k, nh);
    const int nasc = tb.nasc[k], nd = nh - nasc;
    const int* H = tb.hits + (size_t)k * kMaxTlHits;
    const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    int m = 0, prev = -1000;
    for (int j = 0; j < nh; ++j) {
      const int i = (j < nd) ? (nh - 1 - j) : (j - nd);
      if (!key.owns(o, H[i])) continue;
      const int row = Rw[i];
      if (m > 0 && row - prev - 1 > kMaxMiss) {
        if (m >= kMinHits) { ++cs; ch += m; }
        m = 0;
      }
      ++m;
      prev = row;
    }
    if (m >= kMinHits) { ++cs; ch += m; }
  }
  nSeg[k] = cs;
  nSegHits[k] = ch;
}

// K8c: write the sector tracks of each tracklet (ids in tracklet order).
// Hits go straight to their output slots: a segment that turns out too short
// is overwritten by the next kept one, or lies past the tracklet's last kept
// hit and is not written (the slots of a tracklet are exactly its kept hits).
__global__ void __launch_bounds__(128) k_segments_write(const int* __restrict__ nTlDev, OwnCtx o, TrackletBufs tb,
                                                        const int* __restrict__ segPos,
                                                        const int* __restrict__ segHitPos,
                                                        const int2* __restrict__ syz,
                                                        const int* __restrict__ sorig, SectorTrackBufs sb, int capSt,
                                                        int capHits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nTlDev) return;
  const int nh = tb.nhits[k];
  if (nh < kMinHits || segPos[k + 1] == segPos[k]) return;
  const TlKey key = tl_key(o, tb, k, nh);
  const int nasc = tb.nasc[k], nd = nh - nasc;
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
  const int ts = tb.rbase[k] / kNRow;
  const int tf = ts / kNSec, sector = ts % kNSec;
  // the slots end at the tracklet's last kept hit, and at the capacity
  const int hoEnd = min(segHitPos[k + 1], capHits);
  int id = segPos[k], ho = segHitPos[k];
  int m = 0, prev = -1000, first = -1;
  auto flush = [&](void) {
    if (m >= kMinHits) {
      if (id < capSt) {
        sb.tl[id] = k;
        sb.tf[id] = tf;
        sb.sector[id] = sector;
        sb.off[id] = min(ho, capHits);
        sb.zref[id] = syz[first].y;
      }
      ++id;
      ho += m;
    }
    m = 0;
  };
  for (int j = 0; j < nh; ++j) {
    const int i = (j < nd) ? (nh - 1 - j) : (j - nd);
    const int h = H[i];
    if (!key.owns(o, h)) continue;
    const int row = Rw[i];
    if (m > 0 && row - prev - 1 > kMaxMiss) flush();
    if (m == 0) first = h;
    if (ho + m < hoEnd) {
      sb.hits[ho + m] = h;
      sb.rows[ho + m] = (uint8_t)row;
    }
    ++m;
    prev = row;
  }
  flush();
}

// K8d: coordinates and input index of every sector-track hit, gathered once
// (one thread per hit) for the sector fits and the final refit.
__global__ void k_st_gather(const int* __restrict__ nHitsDev, SectorTrackBufs sb, const int2* __restrict__ syz,
                            const int* __restrict__ sorig) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *nHitsDev) return;
  const int h = sb.hits[i];
  sb.yz[i] = syz[h];
  sb.orig[i] = sorig[h];
}

__global__ void __launch_bounds__(128) k_sector_fit(const int* __restrict__ nStDev, TrackletBufs tb,
                                                    const int2* __restrict__ syz, const GeomConst* __restrict__ G,
                                                    SectorTrackBufs sb) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= *nStDev) return;
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  const int b = sb.off[id], m = sb.off[id + 1] - b;
  const int2* P = sb.yz + b;
  const uint8_t* Rw = sb.rows + b;
  const int zref = sb.zref[id];
  KState<float> sd;
  load_state(sd, tb.state + (size_t)sb.tl[id] * 21);
  const float xa = G->rowx[Rw[0]];
  {
    KState<float> tmp = sd;
    if (kf_prop<float>(tmp, xa, bzc) == 0) sd = tmp;
  }
  KState<float> t;
  int2 p = P[0];
  const int yref = p.x;
  kf_reset<float>(t, xa, hit_y(p.x, yref), hit_z(p.y, zref, zunit), sd.p[2], sd.p[3], sd.p[4]);
  for (int i = 1; i < m; ++i) {
    if (kf_prop<float>(t, G->rowx[Rw[i]], bzc) != 0) continue;
    p = P[i];
    kf_update<float>(t, hit_y(p.x, yref), hit_z(p.y, zref, zunit), nullptr);
  }
  store_state(sb.out + (size_t)id * 21, t, yref);
  KState<float> u;
  p = P[m - 1];
  kf_reset<float>(u, G->rowx[Rw[m - 1]], hit_y(p.x, yref), hit_z(p.y, zref, zunit), t.p[2], t.p[3], t.p[4]);
  for (int i = m - 2; i >= 0; --i) {
    if (kf_prop<float>(u, G->rowx[Rw[i]], bzc) != 0) continue;
    p = P[i];
    kf_update<float>(u, hit_y(p.x, yref), hit_z(p.y, zref, zunit), nullptr);
  }
  store_state(sb.in + (size_t)id * 21, u, yref);
}

// ------------------------------------------------------------- launchers
namespace {
struct PassGrid {
  int sms = 0, chain = 0, out = 0, refit = 0, in = 0;
};
PassGrid pass_grid() {
  static PassGrid g;
  if (g.sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.chain, k_tl_chain, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.out, k_tl_out, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.refit, k_tl_refit, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.in, k_tl_in, 128, 0);
  }
  return g;
}
}  // namespace

void launch_tracklets(int nTl, const int* nTlDev, int* workCounter, const int* starts, const int* up,
                      const RowGrid* grid, int nRows, const int* cellStart, const int2* syz, const GeomConst* G,
                      TrackletBufs tb, cudaStream_t st, cudaEvent_t* passEnd) {
  auto mark = [&](int i) {
    if (passEnd) cudaEventRecord(passEnd[i], st);
  };
  if (nTl <= 0) {
    for (int i = 0; i < 4; ++i) mark(i);
    return;
  }
  const PassGrid g = pass_grid();
  auto blocks = [&](int perSm) { return std::min((nTl + 127) / 128, g.sms * std::max(perSm, 1)); };
  cudaMemsetAsync(workCounter, 0, 4 * sizeof(int), st);
  k_tl_chain<<<blocks(g.chain), 128, 0, st>>>(nTlDev, workCounter, starts, up, grid, nRows, syz, G, tb);
  mark(0);
  k_tl_out<<<blocks(g.out), 128, 0, st>>>(nTlDev, workCounter + 1, grid, cellStart, syz, G, tb);
  mark(1);
  k_tl_refit<<<blocks(g.refit), 128, 0, st>>>(nTlDev, workCounter + 2, syz, G, tb);
  mark(2);
  k_tl_in<<<blocks(g.in), 128, 0, st>>>(nTlDev, workCounter + 3, grid, cellStart, syz, G, tb);
  mark(3);
  g_launch_count += 4;
}

void launch_ownership(int nTl, const int* nTlDev, int nSec, const RowGrid* grid, const int* starts, TrackletBufs tb,
                      void* w, int* secBegin, int* wide, cudaStream_t st) {
  cudaMemsetAsync(wide, 0, sizeof(int), st);
  k_sector_ranges<<<(nSec + 1 + 127) / 128, 128, 0, st>>>(nSec, grid, starts, nTlDev, secBegin, wide);
  ++g_launch_count;
  if (nTl > 0) {
    k_ownership<<<(nTl + 127) / 128, 128, 0, st>>>(nTlDev, OwnCtx{secBegin, wide, w}, tb);
    ++g_launch_count;
  }
}

void launch_segments_count(int nTl, const int* nTlDev, const int* secBegin, const int* wide, const void* w,
                           TrackletBufs tb, int* nSeg, int* nSegHits, cudaStream_t st) {
  if (nTl > 0) {
    k_segments_count<<<(nTl + 127) / 128, 128, 0, st>>>(nTlDev, OwnCtx{secBegin, wide, const_cast<void*>(w)}, tb,
                                                         nSeg, nSegHits);
    ++g_launch_count;
  }
}

void launch_segments_write(int nTl, const int* nTlDev, const int* secBegin, const int* wide, const void* w,
                           TrackletBufs tb, const int* segPos, const int* segHitPos, const int2* syz,
                           const int* sorig, SectorTrackBufs sb, int capSt, int capHits, cudaStream_t st) {
  if (nTl > 0) {
    k_segments_write<<<(nTl + 127) / 128, 128, 0, st>>>(nTlDev, OwnCtx{secBegin, wide, const_cast<void*>(w)}, tb,
                                                         segPos, segHitPos, syz, sorig, sb, capSt, capHits);
    ++g_launch_count;
  }
}

void launch_st_gather(int nHits, const int* nHitsDev, SectorTrackBufs sb, const int2* syz, const int* sorig,
                      cudaStream_t st) {
  if (nHits > 0) {
    k_st_gather<<<(nHits + 255) / 256, 256, 0, st>>>(nHitsDev, sb, syz, sorig);
    ++g_launch_count;
  }
}

void launch_sector_fit(int nSt, const int* nStDev, const TrackletBufs tb, const int2* syz, const GeomConst* G,
                       SectorTrackBufs sb, cudaStream_t st) {
  if (nSt > 0) {
    k_sector_fit<<<(nSt + 127) / 128, 128, 0, st>>>(nStDev, tb, syz, G, sb);
    ++g_launch_count;
  }
}

}  // namespace o2tpc
