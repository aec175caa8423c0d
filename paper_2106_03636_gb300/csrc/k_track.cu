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

// Row of hit h linked up from a hit on row R: R + 1, or R + 2 when the link
// crosses a missing row (only with row step 2; without it no row is read).
__device__ inline int link_row(const RowGrid* __restrict__ grid, int R, int h, int rowStep2) {
  if (!rowStep2) return R + 1;
  const RowGrid g = grid[R + 1];
  return h < g.start + g.count ? R + 1 : R + 2;
}

__device__ inline int clamp_i(float v) { return (int)fminf(fmaxf(v, -1.0e9f), 1.0e9f); }

__device__ inline void reset_cov(KState<float>& s, int angErr) {
#pragma unroll
  for (int i = 0; i < 15; ++i) s.C[i] = 0.f;
  kf_meas_cov<float>(s, angErr);
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

// Lanes with want = true take consecutive work items from *counter, one
// atomic per warp; returns this lane's item (meaningful where want).  All 32
// lanes must call it.
__device__ inline int warp_take(int* counter, bool want) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(full, want);
  int base = 0;
  if (m) {
    const int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(full, base, leader);
  }
  return base + __popc(m & ((1u << lane) - 1u));
}

// (a) chain fit: seed from the first and third chain hits, then one update
// per chain hit.  A transport failure drops the tracklet.  One thread per
// tracklet, each walking its own chain (a warp-uniform form of this loop,
// one chain hit of every lane per iteration, measured 30 % slower over
// passes a and c together).
__global__ void __launch_bounds__(128) k_tl_chain(const int* __restrict__ nTlDev, int* __restrict__ counter, const int* __restrict__ starts,
                                                  const int* __restrict__ up, const RowGrid* __restrict__ grid,
                                                  int nRows, const int2* __restrict__ syz,
                                                  const GeomConst* __restrict__ G, TrackletBufs tb) {
  const float zunit = G->zunit, bzc = G->bzc;
  const int rs2 = G->rowStep2;
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
    const int zref = a0.y;
    int yref = a0.x;
    tb.zref[k] = zref;
    tb.rbase[k] = R0 - r0;
    const int h1 = up[h0];
    const int R1 = link_row(grid, R0, h1, rs2);
    const int h2 = up[h1];
    const int R2 = link_row(grid, R1, h2, rs2);
    const int2 a2 = syz[h2];
    const float x0 = G->rowx[r0];
    const float dx = (float)(R2 - R0) * G->pitch, dy = hit_y(a2.x, yref) - hit_y(a0.x, yref);
    const float tphi = dy / dx;
    const float s0 = tphi / sqrtf(1.f + tphi * tphi);
    const float t0 = (hit_z(a2.y, zref, zunit) - hit_z(a0.y, zref, zunit)) / sqrtf(dx * dx + dy * dy);
    KState<float> st;
    kf_reset<float>(st, x0, hit_y(a0.x, yref), hit_z(a0.y, zref, zunit), s0, t0, 0.f);
    kf_meas_cov<float>(st, G->angErr);
    H[0] = h0;
    Rw[0] = (uint8_t)r0;
    int nc = 1, hit = h1, prev = r0, Rh = R1;
    bool dropped = false;
    while (hit >= 0 && nc < kMaxTlHits) {
      const int row = r0 + (Rh - R0);
      const int2 hp = syz[hit];  // both loads in flight during the transport
      const int next = up[hit];
      if (kf_prop_row<float>(st, prev, row, G, bzc) != 0) {
        dropped = true;
        break;
      }
      recentre_y(st.p[0], yref, hp.x);
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr, G->angErr);
      H[nc] = hit;
      Rw[nc] = (uint8_t)row;
      ++nc;
      prev = row;
      hit = next;
      if (hit >= 0) Rh = link_row(grid, Rh, hit, rs2);
    }
    tb.nasc[k] = dropped ? 0 : nc;
    tb.yref[k] = yref;
    if (dropped) tb.nhits[k] = 0;
    else store_raw(tb.state + (size_t)k * 21, st);
  }
}

// (c) inward refit from the top hit through every attached hit; a hit whose
// transport fails is skipped.  One thread per tracklet, as in (a).
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
    int yref = tb.yref[k];
    KState<float> st;
    float* S = tb.state + (size_t)k * 21;
    load_state(st, S);
    int srow = Rw[na - 1];
    for (int i = na - 2; i >= 0; --i) {
      const int2 hp = syz[H[i]];
      if (kf_prop_row<float>(st, srow, Rw[i], G, bzc) != 0) continue;
      srow = Rw[i];
      recentre_y(st.p[0], yref, hp.x);
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr, G->angErr);
    }
    tb.yref[k] = yref;
    store_raw(S, st);
  }
}

// --------------------------------------------- following (passes b, d)
// From the row after the chain's top (b, outward) or below its start (d,
// inward), one pad row per step: transport, search the +-3 sigma window of
// the prediction, update with the best hit; stop after kMaxMiss rows without
// a hit, at the row range end, on a transport failure or when |sin phi| >
// kSinFollow.  The state after the last accepted hit is kept (shared memory)
// and is the pass's result.
//
// One persistent kernel per direction, written as one loop in which every
// iteration is one row step of every busy lane: a lane whose tracklet ends
// takes the next one (one atomic per warp for all such lanes), so the
// transport and the update run converged whatever the tracklets' lengths.
// The row search comes in two forms that pick the same hit:
// * per lane: each lane scans the candidate cells of its own window;
// * warp-cooperative: the candidates of all lanes' windows on this step are
//   laid out one after another and scanned 32 at a time by the whole warp
//   (a lane finds the owner of candidate q by a binary search over the
//   warp's exclusive candidate offsets; per owner the smallest key wins).
// Both score a candidate by the same explicitly rounded expression and keep
// the smallest (chi2 bits << 32 | hit) - chi2 >= 0, so its bit pattern orders
// like its value - which is the rule "smallest chi2, then the smaller
// sorted index".

struct SearchPar {
  float y, z, wy, wz, isy2, isz2;
  int yref, zref;
};

// Window of a row search; false: no candidate can pass (empty row, unusable
// window).  The cell rectangle only has to cover the window: one unit of
// slack on each side absorbs the rounding of the float products.
__device__ inline bool search_window(const RowGrid& g, int npads, const KState<float>& s, int yref, int zref,
                                     float izunit, int angErr, SearchPar& P, int& iy0, int& iy1, int& iz0,
                                     int& iz1) {
  if (g.count == 0) return false;
  float vy, vz;
  meas_var<float>(angErr, s, vy, vz);
  const float sy2 = s.C[0] + vy, sz2 = s.C[2] + vz;
  const float wy = 3.f * sqrtf(sy2), wz = 3.f * sqrtf(sz2);
  if (!(wy < 1e4f) || !(wz < 1e4f) || !isfinite(s.p[0]) || !isfinite(s.p[1])) return false;
  const int ylo = yref + clamp_i(floorf((s.p[0] - wy) * 160.f)) - 1;
  const int yhi = yref + clamp_i(ceilf((s.p[0] + wy) * 160.f)) + 1;
  const int zlo = zref + clamp_i(floorf((s.p[1] - wz) * izunit)) - 1;
  const int zhi = zref + clamp_i(ceilf((s.p[1] + wz) * izunit)) + 1;
  if (!cell_range(g, npads, ylo, yhi, zlo, zhi, iy0, iy1, iz0, iz1)) return false;
  P.y = s.p[0];
  P.z = s.p[1];
  P.wy = wy;
  P.wz = wz;
  P.isy2 = 1.f / sy2;
  P.isz2 = 1.f / sz2;
  P.yref = yref;
  P.zref = zref;
  return true;
}

constexpr unsigned long long kNoHit = ~0ull;

// Key of candidate hit h at p against window P, or kNoHit if it fails the
// window or the chi2 cut.  Every operation is rounded explicitly, so the key
// is the same number wherever this is inlined.
__device__ inline unsigned long long cand_key(int h, int2 p, const SearchPar& P, float zunit) {
  const float dy = __fsub_rn(__fmul_rn((float)(p.x - P.yref), 0.00625f), P.y);
  const float dz = __fsub_rn(__fmul_rn((float)(p.y - P.zref), zunit), P.z);
  if (fabsf(dy) > P.wy || fabsf(dz) > P.wz) return kNoHit;
  const float chi = __fadd_rn(__fmul_rn(__fmul_rn(dy, dy), P.isy2), __fmul_rn(__fmul_rn(dz, dz), P.isz2));
  if (chi > kChi2Follow) return kNoHit;
  return ((unsigned long long)__float_as_uint(chi) << 32) | (unsigned)h;
}

// Per-lane search: cell rows [iz0, iz0 + nseg) x columns [iy0, iy1].
__device__ inline unsigned long long lane_search(int nseg, int cellBase, int ny, int iy0, int iy1, int iz0,
                                                 const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                                 const SearchPar& P, float zunit) {
  unsigned long long best = kNoHit;
  for (int j = 0; j < nseg; ++j) {
    const int cb = cellBase + (iz0 + j) * ny;
    const int a = __ldg(cellStart + cb + iy0);
    const int b = __ldg(cellStart + cb + iy1 + 1);
    for (int h = a; h < b; ++h) {
      const unsigned long long key = cand_key(h, __ldg(syz + h), P, zunit);
      if (key < best) best = key;
    }
  }
  return best;
}

// Warp-cooperative search.  Lane l searches cell rows [iz0, iz0 + nseg) x
// columns [iy0, iy1] of its window sp[l] when nseg > 0; returns its best key.
// All 32 lanes must call it.  sp / sbest: this warp's 32 slots.
__device__ inline unsigned long long coop_search(int nseg, int cellBase, int ny, int iy0, int iy1, int iz0,
                                                 const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                                 const SearchPar* sp, unsigned long long* sbest, float zunit) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  sbest[lane] = kNoHit;
  const int maxseg = (int)__reduce_max_sync(full, (unsigned)nseg);
  __syncwarp();
  for (int j = 0; j < maxseg; ++j) {
    int a = 0, c = 0;
    if (j < nseg) {
      const int cb = cellBase + (iz0 + j) * ny;
      a = __ldg(cellStart + cb + iy0);
      c = __ldg(cellStart + cb + iy1 + 1) - a;
    }
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, inc, o);
      if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(full, inc, 31);
    const int exc = inc - c;
    for (int base = 0; base < total; base += 32) {
      const int q = base + lane;
      // owner: the last lane whose candidates start at or before q
      int own = 0, eown = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int e = __shfl_sync(full, exc, own + step);
        if (e <= q) {
          own += step;
          eown = e;
        }
      }
      const int aown = __shfl_sync(full, a, own);
      unsigned long long key = kNoHit;
      if (q < total) {
        const int h = aown + (q - eown);
        key = cand_key(h, __ldg(syz + h), sp[own], zunit);
      } else {
        own = 32;  // past the end: a run of its own
      }
      // minimum over each run of equal owners (the runs are contiguous)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_down_sync(full, key, o);
        const int ow = __shfl_down_sync(full, own, o);
        if (lane + o < 32 && ow == own && v < key) key = v;
      }
      const int prevOwn = __shfl_up_sync(full, own, 1);
      if (own < 32 && (lane == 0 || prevOwn != own) && key < sbest[own]) sbest[own] = key;
      __syncwarp();
    }
  }
  __syncwarp();
  return sbest[lane];
}

// (b) kDir = +1: outward following above the chain; its result is the
// inward refit's starting state: the last accepted state with the position
// of the top hit and a fresh covariance.  (d) kDir = -1: inward following
// below the chain start; the state kept is the one at the innermost accepted
// hit.  coop: 1 warp-cooperative search, 0 per-lane search.
// Blocks of 128 per SM the following kernels are compiled for: 7 (72
// registers, no spills) measured 2 % faster over both passes on the full
// Time Frame than 8 (64 registers, ~40 bytes of spills).
#ifndef O2TPC_FOLLOW_MIN_BLOCKS
#define O2TPC_FOLLOW_MIN_BLOCKS 7
#endif

template <int kDir>
__global__ void __launch_bounds__(128, O2TPC_FOLLOW_MIN_BLOCKS) k_tl_follow(const int* __restrict__ nTlDev, int* __restrict__ counter,
                                                     const RowGrid* __restrict__ grid,
                                                     const int* __restrict__ cellStart,
                                                     const int2* __restrict__ syz,
                                                     const GeomConst* __restrict__ G, TrackletBufs tb, int coop) {
  __shared__ float s_last[21][128];
  __shared__ SearchPar s_par[128];
  __shared__ unsigned long long s_best[128];
  const unsigned full = 0xffffffffu;
  const int wb = threadIdx.x & ~31;
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  const int nTl = *nTlDev;
  auto save_last = [&](const KState<float>& q) {
    s_last[0][threadIdx.x] = q.x;
#pragma unroll
    for (int j = 0; j < 5; ++j) s_last[1 + j][threadIdx.x] = q.p[j];
#pragma unroll
    for (int j = 0; j < 15; ++j) s_last[6 + j][threadIdx.x] = q.C[j];
  };
  bool have = false, exhausted = false;
  int k = 0, r = 0, n = 0, misses = 0, srow = 0, yref = 0, yrefLast = 0, zref = 0, Rs = 0;
  KState<float> st;
  // ends the lane's tracklet with the state after its last accepted hit
  auto finish = [&]() {
    st.x = s_last[0][threadIdx.x];
#pragma unroll
    for (int j = 0; j < 5; ++j) st.p[j] = s_last[1 + j][threadIdx.x];
#pragma unroll
    for (int j = 0; j < 15; ++j) st.C[j] = s_last[6 + j][threadIdx.x];
    yref = yrefLast;
    float* S = tb.state + (size_t)k * 21;
    if (kDir > 0) {
      const int2 p = syz[tb.hits[(size_t)k * kMaxTlHits + n - 1]];  // the top hit
      recentre_y(st.p[0], yref, p.x);
      st.p[0] = hit_y(p.x, yref);
      st.p[1] = hit_z(p.y, zref, zunit);
      reset_cov(st, G->angErr);
      tb.nasc[k] = n;
      tb.yref[k] = yref;
      store_raw(S, st);
    } else {
      tb.nhits[k] = n;
      store_state(S, st, yref);
    }
    have = false;
  };
  for (;;) {
    // lanes without a tracklet take the next ones
    const bool want = !have && !exhausted;
    const int kk = warp_take(counter, want);
    {
      if (want) {
        k = kk;
        if (k >= nTl) {
          exhausted = true;
        } else {
          const int na = tb.nasc[k];
          if (na > 0) {
            const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
            Rs = tb.rbase[k];
            zref = tb.zref[k];
            yref = tb.yref[k];
            load_state(st, tb.state + (size_t)k * 21);
            n = na;
            r = (kDir > 0) ? Rw[na - 1] + 1 : Rw[0] - 1;
            misses = 0;
            srow = row_of_x(st.x);
            save_last(st);
            yrefLast = yref;
            have = true;
          }
        }
      }
    }
    if (__ballot_sync(full, have) == 0) {
      if (__all_sync(full, exhausted)) break;
      continue;
    }
    // one row step of every busy lane: transport, then the window
    int nseg = 0, cellBase = 0, ny = 0, iy0 = 0, iy1 = 0, iz0 = 0, iz1 = 0;
    SearchPar P;
    if (have) {
      if ((kDir > 0) ? (r >= kNRow) : (r < 0)) {
        finish();
      } else if (kf_prop_row<float>(st, srow, r, G, bzc) != 0 || fabsf(st.p[2]) > kSinFollow) {
        finish();
      } else {
        srow = r;
        const RowGrid g = grid[Rs + r];
        if (search_window(g, G->npads[r], st, yref, zref, izunit, G->angErr, P, iy0, iy1, iz0, iz1)) {
          nseg = iz1 - iz0 + 1;
          cellBase = g.cellBase;
          ny = g.ny;
        }
      }
    }
    unsigned long long best;
    if (coop) {
      if (nseg > 0) s_par[threadIdx.x] = P;
      __syncwarp();
      best = coop_search(nseg, cellBase, ny, iy0, iy1, iz0, cellStart, syz, s_par + wb, s_best + wb, zunit);
    } else {
      best = lane_search(nseg, cellBase, ny, iy0, iy1, iz0, cellStart, syz, P, zunit);
    }
    if (have) {
      if (best != kNoHit) {
        const int hit = (int)(unsigned)(best & 0xffffffffull);
        const int2 hp = syz[hit];
        recentre_y(st.p[0], yref, hp.x);
        kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr, G->angErr);
        tb.hits[(size_t)k * kMaxTlHits + n] = hit;
        tb.rows[(size_t)k * kMaxTlHits + n] = (uint8_t)r;
        ++n;
        save_last(st);
        yrefLast = yref;
        misses = 0;
        r += kDir;
      } else if (++misses >= kMaxMiss) {
        finish();
      } else {
        r += kDir;
      }
    }
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

// Slots [0, 8) of a tracklet's hit list from a 16-byte aligned address (a
// tracklet's 152 slots start on 608-byte boundaries).  Slots past the
// tracklet's hits hold stale values that the callers mask.
__device__ inline void load_hits8(const int* H, int (&hh)[8]) {
  const int4 a = reinterpret_cast<const int4*>(H)[0], b = reinterpret_cast<const int4*>(H)[1];
  hh[0] = a.x; hh[1] = a.y; hh[2] = a.z; hh[3] = a.w;
  hh[4] = b.x; hh[5] = b.y; hh[6] = b.z; hh[7] = b.w;
}

// Ownership bits of slots [0, nh) of a tracklet into this thread's column of
// own[5][128] (bit i % 32 of word i / 32 set: slot i's hit is owned by it).
__device__ inline void owned_bits(const OwnCtx& o, const TlKey& key, const int* H, int nh, unsigned (*own)[128]) {
  for (int i = 0; i < nh; i += 8) {
    int hh[8];
    load_hits8(H + i, hh);
    bool ok[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) ok[u] = (i + u < nh) && key.owns(o, hh[u]);
    unsigned bits = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) bits |= (unsigned)ok[u] << u;
    if ((i & 31) == 0) own[i >> 5][threadIdx.x] = bits;
    else own[i >> 5][threadIdx.x] |= bits << (i & 31);
  }
}
__device__ inline bool is_owned(const unsigned (*own)[128], int i) { return (own[i >> 5][threadIdx.x] >> (i & 31)) & 1u; }

// K8a: hit ownership (atomicMax of the key; a hit already holding a larger
// key is skipped without an atomic).
__global__ void k_ownership(const int* __restrict__ nTlDev, OwnCtx o, TrackletBufs tb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nTlDev) return;
  const int nh = tb.nhits[k];
  if (nh < kMinHits) return;
  const TlKey key = tl_key(o, tb, k, nh);
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  // 8 hits per step (two 16-byte loads; the 152 slots are a multiple of 8),
  // their 8 ownership words loaded before the first atomic
  for (int i = 0; i < nh; i += 8) {
    int hh[8];
    load_hits8(H + i, hh);
    if (key.wide) {
      auto* w = static_cast<unsigned long long*>(o.w);
      unsigned long long v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (i + u < nh) ? w[hh[u]] : ~0ull;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (v[u] < key.k64) atomicMax(&w[hh[u]], key.k64);
    } else {
      auto* w = static_cast<unsigned*>(o.w);
      unsigned v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (i + u < nh) ? w[hh[u]] : ~0u;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (v[u] < key.k32) atomicMax(&w[hh[u]], key.k32);
    }
  }
}

// K8b: segments per tracklet (count pass): owned hits in row order, split at
// gaps of more than kMaxMiss rows, segments of >= kMinHits kept.
__global__ void __launch_bounds__(128) k_segments_count(const int* __restrict__ nTlDev, OwnCtx o, TrackletBufs tb,
                                                        int* __restrict__ nSeg, int* __restrict__ nSegHits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *nTlDev) return;
  __shared__ unsigned s_own[(kMaxTlHits + 31) / 32][128];
  const int nh = tb.nhits[k];
  int cs = 0, ch = 0;
  if (nh >= kMinHits) {
    const TlKey key = tl_key(o, tb, k, nh);
    const int nasc = tb.nasc[k], nd = nh - nasc;
    const int* H = tb.hits + (size_t)k * kMaxTlHits;
    const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    owned_bits(o, key, H, nh, s_own);
    int m = 0, prev = -1000;
    for (int j = 0; j < nh; ++j) {
      const int i = (j < nd) ? (nh - 1 - j) : (j - nd);
      if (!is_owned(s_own, i)) continue;
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
  __shared__ unsigned s_own[(kMaxTlHits + 31) / 32][128];
  const TlKey key = tl_key(o, tb, k, nh);
  const int nasc = tb.nasc[k], nd = nh - nasc;
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
  owned_bits(o, key, H, nh, s_own);
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
    if (!is_owned(s_own, i)) continue;
    const int h = H[i];
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
                                                    SectorTrackBufs sb, const int* __restrict__ order) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= *nStDev) return;
  const int id = order[j];
  const float zunit = G->zunit, bzc = G->bzc;
  const int b = sb.off[id], m = sb.off[id + 1] - b;
  const int2* P = sb.yz + b;
  const uint8_t* Rw = sb.rows + b;
  const int zref = sb.zref[id];
  KState<float> sd;
  load_state(sd, tb.state + (size_t)sb.tl[id] * 21);
  const float xa = G->rowx[Rw[0]];
  {
    KState<float> tmp = sd;
    if (kf_prop_row<float>(tmp, row_of_x(sd.x), Rw[0], G, bzc) == 0) sd = tmp;
  }
  KState<float> t;
  int2 p = P[0];
  int yref = p.x;
  kf_reset<float>(t, xa, hit_y(p.x, yref), hit_z(p.y, zref, zunit), sd.p[2], sd.p[3], sd.p[4]);
  kf_meas_cov<float>(t, G->angErr);
  int srow = Rw[0], zcur = zref;
  for (int i = 1; i < m; ++i) {
    if (kf_prop_row<float>(t, srow, Rw[i], G, bzc) != 0) continue;
    srow = Rw[i];
    p = P[i];
    recentre_y(t.p[0], yref, p.x);
    recentre_z(t.p[1], zcur, p.y, zunit);
    kf_update<float>(t, hit_y(p.x, yref), 0.f, nullptr, G->angErr);
  }
  t.p[1] += (float)(zcur - zref) * zunit;
  store_state(sb.out + (size_t)id * 21, t, yref);
  KState<float> u;
  p = P[m - 1];
  yref = p.x;
  kf_reset<float>(u, G->rowx[Rw[m - 1]], hit_y(p.x, yref), hit_z(p.y, zref, zunit), t.p[2], t.p[3], t.p[4]);
  kf_meas_cov<float>(u, G->angErr);
  srow = Rw[m - 1];
  zcur = P[m - 1].y;
  u.p[1] = 0.f;
  for (int i = m - 2; i >= 0; --i) {
    if (kf_prop_row<float>(u, srow, Rw[i], G, bzc) != 0) continue;
    srow = Rw[i];
    p = P[i];
    recentre_y(u.p[0], yref, p.x);
    recentre_z(u.p[1], zcur, p.y, zunit);
    kf_update<float>(u, hit_y(p.x, yref), 0.f, nullptr, G->angErr);
  }
  u.p[1] += (float)(zcur - zref) * zunit;
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.out, k_tl_follow<1>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.refit, k_tl_refit, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.in, k_tl_follow<-1>, 128, 0);
  }
  return g;
}
}  // namespace

void launch_tracklets(int nTl, const int* nTlDev, int* workCounter, const int* starts, const int* up,
                      const RowGrid* grid, int nRows, const int* cellStart, const int2* syz, const GeomConst* G,
                      TrackletBufs tb, cudaStream_t st, cudaEvent_t* passEnd, bool coopSearch) {
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
  const int coop = coopSearch ? 1 : 0;
  k_tl_follow<1><<<blocks(g.out), 128, 0, st>>>(nTlDev, workCounter + 1, grid, cellStart, syz, G, tb, coop);
  mark(1);
  k_tl_refit<<<blocks(g.refit), 128, 0, st>>>(nTlDev, workCounter + 2, syz, G, tb);
  mark(2);
  k_tl_follow<-1><<<blocks(g.in), 128, 0, st>>>(nTlDev, workCounter + 3, grid, cellStart, syz, G, tb, coop);
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
                       SectorTrackBufs sb, const int* order, cudaStream_t st) {
  if (nSt > 0) {
    k_sector_fit<<<(nSt + 127) / 128, 128, 0, st>>>(nStDev, tb, syz, G, sb, order);
    ++g_launch_count;
  }
}

}  // namespace o2tpc
