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
__device__ inline void load_state(KState<float>& s, const float* src) {
  s.x = src[0];
#pragma unroll
  for (int i = 0; i < 5; ++i) s.p[i] = src[1 + i];
#pragma unroll
  for (int i = 0; i < 15; ++i) s.C[i] = src[6 + i];
}

// K7: persistent threads, one tracklet at a time each, taking the next start
// hit from a global counter as soon as the previous tracklet is done (no lane
// idles until the longest tracklet of its warp ends).  The passes of a
// tracklet (chain fit, outward following, inward refit of the attached hits,
// inward following below the chain) are phases of one loop whose body holds a
// single transport, search and update: threads of a warp in different phases
// still issue the same instructions.  Results do not depend on which thread
// builds which tracklet.
__global__ void __launch_bounds__(128, 6) k_tracklets(int nTl, int* __restrict__ workCounter,
                                                      const int* __restrict__ starts,
                                                      const int* __restrict__ up, const RowGrid* __restrict__ grid,
                                                      int nRows, const int* __restrict__ cellStart,
                                                      const int2* __restrict__ syz, const GeomConst* __restrict__ G,
                                                      TrackletBufs tb) {
  // the state after the last accepted hit lives in shared memory (one column
  // per thread) rather than in registers
  __shared__ float s_last[21][128];
  auto save_last = [&](const KState<float>& q) {
    s_last[0][threadIdx.x] = q.x;
#pragma unroll
    for (int j = 0; j < 5; ++j) s_last[1 + j][threadIdx.x] = q.p[j];
#pragma unroll
    for (int j = 0; j < 15; ++j) s_last[6 + j][threadIdx.x] = q.C[j];
  };
  auto load_last = [&](KState<float>& q) {
    q.x = s_last[0][threadIdx.x];
#pragma unroll
    for (int j = 0; j < 5; ++j) q.p[j] = s_last[1 + j][threadIdx.x];
#pragma unroll
    for (int j = 0; j < 15; ++j) q.C[j] = s_last[6 + j][threadIdx.x];
  };
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  // phases: 0 chain fit, 1 outward following, 2 inward refit, 3 inward
  // following, 5 take the next tracklet
  int phase = 5, k = 0, r0 = 0, Rs = 0, zref = 0, yref = 0;
  int i = 0, r = 0, nc = 0, na = 0, nd = 0, misses = 0, top = 0, chainHit = -1;
  int* H = nullptr;
  uint8_t* Rw = nullptr;
  KState<float> st;
  // end of the outward following: restart at the top hit, fresh covariance
  auto begin_refit = [&]() {
    load_last(st);
    const int2 p = syz[top];
    st.p[0] = hit_y(p.x, yref);
    st.p[1] = hit_z(p.y, zref, zunit);
    reset_cov(st);
    i = na - 2;
    phase = 2;
  };
  auto finish = [&](bool dropped) {
    if (dropped) {
      tb.nhits[k] = 0;
      tb.nasc[k] = 0;
    } else {
      tb.nhits[k] = na + nd;
      tb.nasc[k] = na;
      load_last(st);
      store_state(tb.state + (size_t)k * 21, st, yref);
    }
    phase = 5;
  };
  for (;;) {
    if (phase == 5) {
      k = atomicAdd(workCounter, 1);
      if (k >= nTl) break;
      const int h0 = starts[k];
      const int R0 = find_row(grid, nRows, h0);
      r0 = (R0 % kRowsPerTF) % kNRow;
      Rs = R0 - r0;
      H = tb.hits + (size_t)k * kMaxTlHits;
      Rw = tb.rows + (size_t)k * kMaxTlHits;
      const int2 a0 = syz[h0];
      zref = a0.y;
      yref = a0.x;
      tb.zref[k] = zref;
      const int h1 = up[h0];
      const int2 a2 = syz[up[h1]];
      const float x0 = G->rowx[r0], x2 = G->rowx[r0 + 2];
      const float dx = x2 - x0, dy = hit_y(a2.x, yref) - hit_y(a0.x, yref);
      const float tphi = dy / dx;
      const float s0 = tphi / sqrtf(1.f + tphi * tphi);
      const float t0 = (hit_z(a2.y, zref, zunit) - hit_z(a0.y, zref, zunit)) / sqrtf(dx * dx + dy * dy);
      kf_reset<float>(st, x0, hit_y(a0.x, yref), hit_z(a0.y, zref, zunit), s0, t0, 0.f);
      H[0] = h0;
      Rw[0] = (uint8_t)r0;
      nc = 1;
      chainHit = h1;
      nd = 0;
      misses = 0;
      phase = 0;
      continue;
    }
    int row, hit = -1, nextChain = -1;
    int2 hp = make_int2(0, 0);  // coordinates of the hit to add
    bool search = false;
    if (phase == 0) {
      if (chainHit < 0 || nc >= kNRow - r0) {
        na = nc;
        top = H[nc - 1];
        save_last(st);
        r = r0 + nc;
        misses = 0;
        phase = 1;
        continue;
      }
      row = r0 + nc;
      hit = chainHit;
      // both loads in flight during the transport
      hp = syz[hit];
      nextChain = up[hit];
    } else if (phase == 1) {
      if (r >= kNRow) {
        begin_refit();
        continue;
      }
      row = r;
      search = true;
    } else if (phase == 2) {
      if (i < 0) {
        save_last(st);
        r = r0 - 1;
        misses = 0;
        phase = 3;
        continue;
      }
      row = Rw[i];
      hit = H[i];
      hp = syz[hit];
    } else {
      if (r < 0) {
        finish(false);
        continue;
      }
      row = r;
      search = true;
    }
    bool stop = kf_prop<float>(st, G->rowx[row], bzc) != 0;
    if (!stop && search) {
      stop = fabsf(st.p[2]) > kSinFollow;
      if (!stop) hit = search_row(grid[Rs + row], G->npads[row], cellStart, syz, st, yref, zref, zunit, izunit, &hp);
    }
    if (stop) {
      if (phase == 0) finish(true);
      else if (phase == 2) --i;
      else if (phase == 1) begin_refit();
      else finish(false);
      continue;
    }
    if (hit >= 0) {
      kf_update<float>(st, hit_y(hp.x, yref), hit_z(hp.y, zref, zunit), nullptr);
      if (phase == 0) {
        H[nc] = hit;
        Rw[nc] = (uint8_t)row;
        ++nc;
        chainHit = nextChain;
      } else if (phase == 1) {
        H[na] = hit;
        Rw[na] = (uint8_t)row;
        ++na;
        top = hit;
        save_last(st);
        misses = 0;
      } else if (phase == 3) {
        H[na + nd] = hit;
        Rw[na + nd] = (uint8_t)row;
        ++nd;
        save_last(st);
        misses = 0;
      }
    } else if (search && ++misses >= kMaxMiss) {
      if (phase == 1) begin_refit();
      else finish(false);
      continue;
    }
    if (phase == 1) ++r;
    else if (phase == 2) --i;
    else if (phase == 3) --r;
  }
}

__device__ inline int tf_of(const int* __restrict__ begin, int nTF, int k) {
  return upper_bound_i32(begin, nTF + 1, k) - 1;
}

__device__ inline unsigned long long own_key(int nh, int kl) {
  return ((unsigned long long)(unsigned)nh << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)kl);
}

// K8a: hit ownership.
__global__ void k_ownership(int nTl, const int* __restrict__ tlTfBegin, int nTF, TrackletBufs tb,
                            unsigned long long* __restrict__ w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nTl) return;
  const int nh = tb.nhits[k];
  if (nh < kMinHits) return;
  const int tf = tf_of(tlTfBegin, nTF, k);
  const unsigned long long key = own_key(nh, k - tlTfBegin[tf]);
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  for (int i = 0; i < nh; ++i) atomicMax(&w[H[i]], key);
}

// K8b: segments per tracklet (count pass).  Segment buffers live in local
// memory (at most one hit per row).
__global__ void __launch_bounds__(128) k_segments_count(int nTl, const int* __restrict__ tlTfBegin, int nTF,
                                                        TrackletBufs tb, const unsigned long long* __restrict__ w,
                                                        int* __restrict__ nSeg, int* __restrict__ nSegHits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nTl) return;
  const int nh = tb.nhits[k];
  int cs = 0, ch = 0;
  if (nh >= kMinHits) {
    const int tf = tf_of(tlTfBegin, nTF, k);
    const unsigned long long key = own_key(nh, k - tlTfBegin[tf]);
    const int nasc = tb.nasc[k], nd = nh - nasc;
    const int* H = tb.hits + (size_t)k * kMaxTlHits;
    const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
    int m = 0, prev = -1000;
    for (int j = 0; j < nh; ++j) {
      const int i = (j < nd) ? (nh - 1 - j) : (j - nd);
      if (w[H[i]] != key) continue;
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
// A segment is staged in local memory and written only if it is kept.
__global__ void __launch_bounds__(128) k_segments_write(int nTl, const int* __restrict__ tlTfBegin, int nTF,
                                                        TrackletBufs tb, const unsigned long long* __restrict__ w,
                                                        const int* __restrict__ segPos,
                                                        const int* __restrict__ segHitPos,
                                                        const int2* __restrict__ syz, const RowGrid* __restrict__ grid,
                                                        int nRows, SectorTrackBufs sb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nTl) return;
  const int nh = tb.nhits[k];
  if (nh < kMinHits || segPos[k + 1] == segPos[k]) return;
  const int tf = tf_of(tlTfBegin, nTF, k);
  const unsigned long long key = own_key(nh, k - tlTfBegin[tf]);
  const int nasc = tb.nasc[k], nd = nh - nasc;
  const int* H = tb.hits + (size_t)k * kMaxTlHits;
  const uint8_t* Rw = tb.rows + (size_t)k * kMaxTlHits;
  const int sector = (find_row(grid, nRows, H[0]) % kRowsPerTF) / kNRow;
  int seg[kNRow];
  uint8_t segRow[kNRow];
  int id = segPos[k], ho = segHitPos[k];
  int m = 0, prev = -1000;
  auto flush = [&](void) {
    if (m >= kMinHits) {
      for (int q = 0; q < m; ++q) {
        sb.hits[ho + q] = seg[q];
        sb.rows[ho + q] = segRow[q];
      }
      sb.tl[id] = k;
      sb.tf[id] = tf;
      sb.sector[id] = sector;
      sb.off[id] = ho;
      sb.zref[id] = syz[seg[0]].y;
      ++id;
      ho += m;
    }
    m = 0;
  };
  for (int j = 0; j < nh; ++j) {
    const int i = (j < nd) ? (nh - 1 - j) : (j - nd);
    const int h = H[i];
    if (w[h] != key) continue;
    const int row = Rw[i];
    if (m > 0 && row - prev - 1 > kMaxMiss) flush();
    seg[m] = h;
    segRow[m] = (uint8_t)row;
    ++m;
    prev = row;
  }
  flush();
}

// K8d: outward then inward fit of every sector track.  The outward fit seeds
// (sin phi, t, q/pT) from the tracklet's state moved to the first hit; the
// inward fit seeds them from the outward result.
__global__ void __launch_bounds__(128) k_sector_fit(int nSt, TrackletBufs tb, const int2* __restrict__ syz,
                                                    const GeomConst* __restrict__ G, SectorTrackBufs sb) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nSt) return;
  const float zunit = G->zunit, izunit = G->kz, bzc = G->bzc;
  const int b = sb.off[id], m = sb.off[id + 1] - b;
  const int* H = sb.hits + b;
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
  int2 p = syz[H[0]];
  const int yref = p.x;
  kf_reset<float>(t, xa, hit_y(p.x, yref), hit_z(p.y, zref, zunit), sd.p[2], sd.p[3], sd.p[4]);
  for (int i = 1; i < m; ++i) {
    if (kf_prop<float>(t, G->rowx[Rw[i]], bzc) != 0) continue;
    p = syz[H[i]];
    kf_update<float>(t, hit_y(p.x, yref), hit_z(p.y, zref, zunit), nullptr);
  }
  store_state(sb.out + (size_t)id * 21, t, yref);
  KState<float> u;
  p = syz[H[m - 1]];
  kf_reset<float>(u, G->rowx[Rw[m - 1]], hit_y(p.x, yref), hit_z(p.y, zref, zunit), t.p[2], t.p[3], t.p[4]);
  for (int i = m - 2; i >= 0; --i) {
    if (kf_prop<float>(u, G->rowx[Rw[i]], bzc) != 0) continue;
    p = syz[H[i]];
    kf_update<float>(u, hit_y(p.x, yref), hit_z(p.y, zref, zunit), nullptr);
  }
  store_state(sb.in + (size_t)id * 21, u, yref);
}

// ------------------------------------------------------------- launchers
void launch_tracklets(int nTl, int* workCounter, const int* starts, const int* up, const RowGrid* grid, int nRows,
                      const int* cellStart, const int2* syz, const GeomConst* G, TrackletBufs tb, cudaStream_t st) {
  if (nTl <= 0) return;
  static int sms = 0, perSm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSm, k_tracklets, 128, 0);
    if (perSm < 1) perSm = 1;
  }
  const int blocks = std::min((nTl + 127) / 128, sms * perSm);
  cudaMemsetAsync(workCounter, 0, sizeof(int), st);
  k_tracklets<<<blocks, 128, 0, st>>>(nTl, workCounter, starts, up, grid, nRows, cellStart, syz, G, tb);
  ++g_launch_count;
}

void launch_ownership(int nTl, const int* tlTfBegin, int nTF, TrackletBufs tb, unsigned long long* w, cudaStream_t st) {
  if (nTl > 0) {
    k_ownership<<<(nTl + 127) / 128, 128, 0, st>>>(nTl, tlTfBegin, nTF, tb, w);
    ++g_launch_count;
  }
}

void launch_segments_count(int nTl, const int* tlTfBegin, int nTF, TrackletBufs tb, const unsigned long long* w,
                           int* nSeg, int* nSegHits, cudaStream_t st) {
  if (nTl > 0) {
    k_segments_count<<<(nTl + 127) / 128, 128, 0, st>>>(nTl, tlTfBegin, nTF, tb, w, nSeg, nSegHits);
    ++g_launch_count;
  }
}

void launch_segments_write(int nTl, const int* tlTfBegin, int nTF, TrackletBufs tb, const unsigned long long* w,
                           const int* segPos, const int* segHitPos, const int2* syz, const RowGrid* grid, int nRows,
                           SectorTrackBufs sb, cudaStream_t st) {
  if (nTl > 0)
    k_segments_write<<<(nTl + 127) / 128, 128, 0, st>>>(nTl, tlTfBegin, nTF, tb, w, segPos, segHitPos, syz, grid,
                                                        nRows, sb);
    ++g_launch_count;
}

void launch_sector_fit(int nSt, const TrackletBufs tb, const int2* syz, const GeomConst* G, SectorTrackBufs sb,
                       cudaStream_t st) {
  if (nSt > 0) {
    k_sector_fit<<<(nSt + 127) / 128, 128, 0, st>>>(nSt, tb, syz, G, sb);
    ++g_launch_count;
  }
}

}  // namespace o2tpc
