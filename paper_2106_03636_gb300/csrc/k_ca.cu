// k_ca.cu - cellular-automaton seeding: NeighboursFinder, NeighboursCleaner,
// StartHitsFinder, plus the device-wide scan used for ordered compaction.
//
// All decisions here are integer: the straightness metric of a hit h with an
// upper neighbour u (row r+1) and a lower neighbour d (row r-1) is
//   D = 2077 (2 y_h - y_u - y_d)^2 + 1536 (2 z_h - z_u - z_d)^2
// (a 2-dof chi2 scaled by 6 sigma_y^2 * 6 sigma_z^2 in integer units; it fits
// in 31 bits inside the windows), accepted when D <= 16 * 1536 * 2077, and
// the winner is the lexicographic minimum of (D, u, d), which no enumeration
// order can change.
#include "o2tpc_kernels.cuh"

namespace o2tpc {

#ifndef O2TPC_NF_CAND
#define O2TPC_NF_CAND 6
#endif
constexpr int kNFCand = O2TPC_NF_CAND;  // candidates per side held in registers by the NeighboursFinder

// Candidate residuals of one side, packed: (y_h - y_c + 1024) << 16 |
// (z_h - z_c + 1024).  Inside the windows both halves stay in [776, 1272], so
// the sum of an up and a down residual adds the halves without carries and
// unpacks to (2 y_h - y_u - y_d + 2048, 2 z_h - z_u - z_d + 2048).
__device__ inline unsigned pack_res(int dy, int dz) { return ((unsigned)(dy + 1024) << 16) | (unsigned)(dz + 1024); }

// Appends the in-window candidates of one side (cells [iy0, iy1] of cell
// rows iz0..iz1 of row g, visited in ascending sorted index) to the register
// slots: the newest goes to slot kNFCand-1, older ones move down, so slots
// [kNFCand - n, kNFCand) hold them in ascending index order.  Returns the
// number found (more than kNFCand: the caller takes the general path).
// pts[c - base] holds the coordinates of sorted hit c (the block's staged
// slab, or the global array with base 0).
__device__ inline int nf_collect(const RowGrid& g, int iy0, int iy1, int iz0, int iz1,
                                 const int* __restrict__ cellStart, const int2* pts, int base, int2 hh,
                                 int (&idx)[kNFCand], unsigned (&res)[kNFCand]) {
  int n = 0;
  for (int iz = iz0; iz <= iz1; ++iz) {
    const int a = __ldg(cellStart + g.cellBase + iz * g.ny + iy0);
    const int b = __ldg(cellStart + g.cellBase + iz * g.ny + iy1 + 1);
    for (int c = a; c < b; ++c) {
      const int2 p = pts[c - base];
      const int dy = hh.x - p.x, dz = hh.y - p.y;
      if (abs(dy) > kWinY || abs(dz) > kWinZ) continue;
#pragma unroll
      for (int q = 0; q < kNFCand - 1; ++q) {
        idx[q] = idx[q + 1];
        res[q] = res[q + 1];
      }
      idx[kNFCand - 1] = c;
      res[kNFCand - 1] = pack_res(dy, dz);
      ++n;
    }
  }
  return n;
}

// K4: one thread per hit; blocks of kB hits tile the rows
// (nfBlockStart, built for the same block size, maps a block to its row,
// looked up once per block).
// --- staging of the adjacent rows' candidate slabs (TMA bulk copy)
constexpr int kSlab = 1024;            // staged hits per side (8 KB)
constexpr int kSlabWaitLimit = 1 << 22;  // mbarrier polls before giving up on a copy

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Injected fault (o2tpc_config.debug_inject bit 0): the barrier is armed for
// the slab bytes but no copy is issued, and the waits give up after this many
// polls - a wait that runs out with nothing in flight.
constexpr int kSlabWaitInjected = 64;

// Waits (bounded) for phase 0 of the mbarrier; false if it did not complete.
__device__ inline bool slab_wait(unsigned bar, int limit) {
  for (int i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// K4: one thread per hit; blocks of kB hits tile the rows (nfBlockStart,
// built for the same block size, maps a block to its row, looked up once per
// block).  With kStage, the candidates come from shared memory: a block's
// hits are consecutive in (cell, input) order, so they lie in the cell rows
// between those of its first and last hit, and their candidates in the cell
// rows of each adjacent pad row that this drift range (widened by the window)
// reaches - every cell across the row, one contiguous range of the sorted
// coordinates.  Thread 0 issues one TMA bulk copy per side as soon as it knows
// the range, completing on an mbarrier; the threads set up their windows
// meanwhile and wait just before scanning.  A side whose range exceeds kSlab
// hits (or a copy that does not complete within the wait limit, flagged in
// err) reads global memory instead.  Without kStage every candidate is a
// global (L1-cached) load.
template <int kB, bool kStage>
__global__ void __launch_bounds__(kB) k_neighbours(const RowGrid* __restrict__ grid,
                                                   const int* __restrict__ nfBlockStart, int nRows,
                                                   const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                                   const GeomConst* __restrict__ G, int* __restrict__ upRaw,
                                                   int* __restrict__ dnRaw, unsigned* __restrict__ err,
                                                   unsigned inject) {
  if ((int)blockIdx.x >= nfBlockStart[nRows]) return;  // launched with an upper bound of blocks
  __shared__ __align__(16) int2 s_slab[kStage ? 2 : 1][kStage ? kSlab : 1];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ int s_row, s_base[2], s_use[2];
  const unsigned bar = smem_addr(&s_bar);
  if (threadIdx.x == 0) {
    const int R0 = upper_bound_i32(nfBlockStart, nRows + 1, blockIdx.x) - 1;
    s_row = R0;
    s_use[0] = s_use[1] = 0;
    const int r0 = (R0 % kRowsPerTF) % kNRow;
    if (kStage && r0 >= 1 && r0 <= kNRow - 2) {
      const RowGrid g0 = grid[R0];
      const int hf = g0.start + (blockIdx.x - nfBlockStart[R0]) * kB;
      const int hl = min(hf + kB, g0.start + g0.count) - 1;
      // drift range of the block's cell rows
      const int izf = cell_iz_floor(syz[hf].y, g0), izl = cell_iz_floor(syz[hl].y, g0);
      const long long zlo = (long long)g0.zmin + (long long)izf * g0.cz - kWinZ;
      const long long zhi = (long long)g0.zmin + (long long)(izl + 1) * g0.cz - 1 + kWinZ;
      unsigned bytes = 0;
      for (int side = 0; side < 2; ++side) {
        const RowGrid g2 = grid[side == 0 ? R0 + 1 : R0 - 1];
        s_base[side] = 0;
        if (g2.count == 0) continue;
        const int zl = (int)max(zlo, (long long)INT_MIN + 1), zh = (int)min(zhi, (long long)INT_MAX - 1);
        int iza = cell_iz_floor(zl, g2), izb = cell_iz_floor(zh, g2);
        if (iza < 0) iza = 0;
        if (izb > g2.nz - 1) izb = g2.nz - 1;
        if (iza > izb) continue;
        const int a = cellStart[g2.cellBase + iza * g2.ny], b = cellStart[g2.cellBase + (izb + 1) * g2.ny];
        const int a0 = a & ~1, b0 = (b + 1) & ~1;  // 16-byte aligned range (syz has one int2 of padding)
        if (b0 - a0 > kSlab || b0 <= a0) continue;
        s_use[side] = b0 - a0;
        s_base[side] = a0;
        bytes += (unsigned)(b0 - a0) * 8u;
      }
      if (bytes) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        for (int side = 0; side < 2; ++side)
          if (s_use[side] && !(inject & 1u))
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(&s_slab[side][0])),
                "l"(syz + s_base[side]), "r"((unsigned)s_use[side] * 8u), "r"(bar)
                : "memory");
      }
    }
  }
  __syncthreads();
  const int R = s_row;
  const RowGrid g = grid[R];
  const int h = g.start + (blockIdx.x - nfBlockStart[R]) * kB + threadIdx.x;
  const bool valid = h < g.start + g.count;
  const int r = (R % kRowsPerTF) % kNRow;
  if (r < 1 || r > kNRow - 2) {  // rows 0 and 151 get no links (no copy was issued)
    if (valid) {
      upRaw[h] = -1;
      dnRaw[h] = -1;
    }
    return;
  }
  const bool staged = kStage && (s_use[0] || s_use[1]);
  const int waitLimit = (inject & 1u) ? kSlabWaitInjected : kSlabWaitLimit;
  bool slabOk = true;
  int bu = -1, bd = -1;
  if (valid) {
    const RowGrid gu = grid[R + 1], gd = grid[R - 1];
    const int npu = G->npads[r + 1], npd = G->npads[r - 1];
    const int2 hh = syz[h];
    const int yh = hh.x, zh = hh.y;
    int uy0, uy1, uz0, uz1, dy0, dy1, dz0, dz1;
    const bool inWin = cell_range(gu, npu, yh - kWinY, yh + kWinY, zh - kWinZ, zh + kWinZ, uy0, uy1, uz0, uz1) &&
                       cell_range(gd, npd, yh - kWinY, yh + kWinY, zh - kWinZ, zh + kWinZ, dy0, dy1, dz0, dz1);
    if (staged) {
      slabOk = slab_wait(bar, waitLimit);
      if (!slabOk) atomicOr(err, kErrTimeout);
    }
    const int2* su = (staged && slabOk && s_use[0]) ? s_slab[0] : syz;
    const int bu0 = (staged && slabOk && s_use[0]) ? s_base[0] : 0;
    const int2* sd = (staged && slabOk && s_use[1]) ? s_slab[kStage ? 1 : 0] : syz;
    const int bd0 = (staged && slabOk && s_use[1]) ? s_base[1] : 0;
    if (inWin) {
      int ui[kNFCand] = {}, di[kNFCand] = {};
      unsigned ur[kNFCand] = {}, dr[kNFCand] = {};
      const int nu = nf_collect(gu, uy0, uy1, uz0, uz1, cellStart, su, bu0, hh, ui, ur);
      const int nd = nu > 0 ? nf_collect(gd, dy0, dy1, dz0, dz1, cellStart, sd, bd0, hh, di, dr) : 0;
      // bestD starts one above the cut, so "D < bestD" also applies the cut
      int bestD = kMaxMetric + 1;
      // pairs in ascending (u, d): a strict "<" keeps the first minimum,
      // which is the lexicographic minimum of (D, u, d).  Slots [a0, kNFCand)
      // of both sides: the last four when both sides fit there (the common
      // case), else all of them.
      auto pair_scan = [&](const int a0) {
#pragma unroll
        for (int a = a0; a < kNFCand; ++a)
#pragma unroll
          for (int b = a0; b < kNFCand; ++b) {
            const unsigned sres = ur[a] + dr[b];
            const int ey = (int)(sres >> 16) - 2048, ez = (int)(sres & 0xFFFFu) - 2048;
            const int D = kWeightY * ey * ey + kWeightZ * ez * ez;
            if (a >= kNFCand - nu && b >= kNFCand - nd && D < bestD) {
              bestD = D;
              bu = ui[a];
              bd = di[b];
            }
          }
      };
      constexpr int kNFSmall = kNFCand < 4 ? kNFCand : 4;
      if (nu <= kNFSmall && nd <= kNFSmall) {
        pair_scan(kNFCand - kNFSmall);
      } else if (nu <= kNFCand && nd <= kNFCand) {
        pair_scan(0);
      } else {
        const int y2 = 2 * yh, z2 = 2 * zh;
        for (int izu = uz0; izu <= uz1; ++izu) {
          const int ua = __ldg(cellStart + gu.cellBase + izu * gu.ny + uy0);
          const int ub = __ldg(cellStart + gu.cellBase + izu * gu.ny + uy1 + 1);
          for (int u = ua; u < ub; ++u) {
            const int2 pu = __ldg(syz + u);
            if (abs(pu.x - yh) > kWinY || abs(pu.y - zh) > kWinZ) continue;
            for (int izd = dz0; izd <= dz1; ++izd) {
              const int da = __ldg(cellStart + gd.cellBase + izd * gd.ny + dy0);
              const int db = __ldg(cellStart + gd.cellBase + izd * gd.ny + dy1 + 1);
              for (int d = da; d < db; ++d) {
                const int2 pd = __ldg(syz + d);
                if (abs(pd.x - yh) > kWinY || abs(pd.y - zh) > kWinZ) continue;
                const int ey = y2 - pu.x - pd.x, ez = z2 - pu.y - pd.y;
                const int D = kWeightY * ey * ey + kWeightZ * ez * ez;
                if (D < bestD) {  // (u, d) visited in ascending order
                  bestD = D;
                  bu = u;
                  bd = d;
                }
              }
            }
          }
        }
      }
    }
  }
  if (valid) {
    upRaw[h] = bu;
    dnRaw[h] = bd;
  }
  // a copy that did not complete in time must land before the block's shared
  // memory is released: thread 0 waits once more (the copies are at most 16 KB
  // of device memory, microseconds against a limit of seconds; with the
  // injected fault nothing was issued, so nothing can land later)
  if (staged && threadIdx.x == 0) slab_wait(bar, waitLimit);
}

// K4b (row step 2, optional): a hit with no accepted pair on the adjacent
// rows may link across one missing row - up on row r + a, down on row r - b,
// (a, b) in {(2,1), (1,2), (2,2)} - with the residual (a + b) h - b u - a d,
// whose variance is f = (a + b)^2 + a^2 + b^2 times a cluster's, so the
// metric D = 2077 e_y^2 + 1536 e_zeta^2 scaled by 6 / f is the same 2-dof
// chi2 (accepted if 6 D <= kMaxMetric f); windows scale with the row
// distance.  The best pair minimises D / f (compared exactly as
// D1 f2 < D2 f1 in 64 bits), ties to the smaller u, then d.  One thread per
// hit; hits that found an adjacent-row pair return at once.
__global__ void k_neighbours_gap(const int* __restrict__ nDev, const RowGrid* __restrict__ grid, int nRows,
                                 const int* __restrict__ cellStart, const int2* __restrict__ syz,
                                 const GeomConst* __restrict__ G, int* __restrict__ upRaw,
                                 int* __restrict__ dnRaw) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= *nDev || upRaw[h] >= 0) return;
  int lo = 0, hi = nRows;  // row of h: the last row starting at or before it
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (grid[m].start <= h) lo = m + 1;
    else hi = m;
  }
  const int R = lo - 1;
  const int r = (R % kRowsPerTF) % kNRow;
  if (r < 1 || r > kNRow - 2) return;
  const int2 hh = syz[h];
  const int yh = hh.x, zh = hh.y;
  long long bD = -1, bf = 1;
  int bu = -1, bd = -1;
  constexpr int kSteps[3][2] = {{2, 1}, {1, 2}, {2, 2}};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int a = kSteps[q][0], b = kSteps[q][1];
    if (r + a > kNRow - 1 || r - b < 0) continue;
    const RowGrid gu = grid[R + a], gd = grid[R - b];
    int uy0, uy1, uz0, uz1, dy0, dy1, dz0, dz1;
    if (!cell_range(gu, G->npads[r + a], yh - a * kWinY, yh + a * kWinY, zh - a * kWinZ, zh + a * kWinZ, uy0, uy1,
                    uz0, uz1))
      continue;
    if (!cell_range(gd, G->npads[r - b], yh - b * kWinY, yh + b * kWinY, zh - b * kWinZ, zh + b * kWinZ, dy0, dy1,
                    dz0, dz1))
      continue;
    const long long f = (long long)((a + b) * (a + b) + a * a + b * b);
    for (int izu = uz0; izu <= uz1; ++izu) {
      const int ua = __ldg(cellStart + gu.cellBase + izu * gu.ny + uy0);
      const int ub = __ldg(cellStart + gu.cellBase + izu * gu.ny + uy1 + 1);
      for (int u = ua; u < ub; ++u) {
        const int2 pu = __ldg(syz + u);
        if (abs(pu.x - yh) > a * kWinY || abs(pu.y - zh) > a * kWinZ) continue;
        for (int izd = dz0; izd <= dz1; ++izd) {
          const int da = __ldg(cellStart + gd.cellBase + izd * gd.ny + dy0);
          const int db = __ldg(cellStart + gd.cellBase + izd * gd.ny + dy1 + 1);
          for (int d = da; d < db; ++d) {
            const int2 pd = __ldg(syz + d);
            if (abs(pd.x - yh) > b * kWinY || abs(pd.y - zh) > b * kWinZ) continue;
            const long long ey = (long long)(a + b) * yh - (long long)b * pu.x - (long long)a * pd.x;
            const long long ez = (long long)(a + b) * zh - (long long)b * pu.y - (long long)a * pd.y;
            const long long D = (long long)kWeightY * ey * ey + (long long)kWeightZ * ez * ez;
            if (6 * D > (long long)kMaxMetric * f) continue;
            const bool better = bu < 0 || D * bf < bD * f || (D * bf == bD * f && (u < bu || (u == bu && d < bd)));
            if (better) {
              bD = D;
              bf = f;
              bu = u;
              bd = d;
            }
          }
        }
      }
    }
  }
  if (bu >= 0) {
    upRaw[h] = bu;
    dnRaw[h] = bd;
  }
}

// K5 + K6a: reciprocity filter on the raw (snapshot) links and the chain-head
// flag: dn < 0, up >= 0, up[up] >= 0 (chains of at least three hits).
__global__ void k_clean(const int* __restrict__ nDev, const int* __restrict__ upRaw, const int* __restrict__ dnRaw,
                        int* __restrict__ up, int* __restrict__ dn, int* __restrict__ startFlag) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= *nDev) return;
  int u = upRaw[h], d = dnRaw[h];
  int uc = (u >= 0 && dnRaw[u] == h) ? u : -1;
  int dc = (d >= 0 && upRaw[d] == h) ? d : -1;
  up[h] = uc;
  dn[h] = dc;
  int flag = 0;
  if (dc < 0 && uc >= 0) {
    int uu = upRaw[uc];
    int uuc = (uu >= 0 && dnRaw[uu] == uc) ? uu : -1;
    flag = uuc >= 0;
  }
  startFlag[h] = flag;
}

// --------------------------------------------------------------- scans
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline int warp_incl(int x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// inclusive block scan for blockDim == 1024; returns the exclusive prefix
__device__ inline int block_excl(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = warp_incl(v);
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) ws[lane] = warp_incl(ws[lane]);
  __syncthreads();
  int incl = x + (w > 0 ? ws[w - 1] : 0);
  if (total) *total = ws[31];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int* __restrict__ in, int nHost,
                                                            const int* __restrict__ nDev, int* __restrict__ sums) {
  const int n = nDev ? *nDev : nHost;
  long long base = (long long)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int tot;
  block_excl(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_mid(int* __restrict__ sums, int nb) {
  int per = (nb + kScanThreads - 1) / kScanThreads;
  int b = threadIdx.x * per, e = min(nb, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += sums[i];
  int off = block_excl(s, nullptr);
  for (int i = b; i < e; ++i) {
    int v = sums[i];
    sums[i] = off;
    off += v;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ in, int nHost,
                                                             const int* __restrict__ nDev, const int* __restrict__ sums,
                                                             int* __restrict__ out) {
  const int n = nDev ? *nDev : nHost;
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + k;
    v[k] = (i < n) ? in[i] : 0;
    s += v[k];
  }
  int tot;
  int off = block_excl(s, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + k;
    if (i < n) out[i] = off;
    off += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = off;
}

// out[0..m] = exclusive scan of in[0..m-1], out[m] = total, m = *nDev <= n
// (the grid covers n; tiles past m add zeros), or m = n when nDev is null;
// out may alias in.
// scratch: >= scan_scratch_ints(n) ints.
int scan_scratch_ints(long long n) { return (int)((n + kScanTile - 1) / kScanTile) + 1; }

__global__ void k_store_zero_at(int* __restrict__ out, int nHost, const int* __restrict__ nDev) {
  out[nDev ? *nDev : nHost] = 0;
}

void scan_exclusive(const int* in, int* out, int n, const int* nDev, int* scratch, cudaStream_t st) {
  int nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    k_store_zero_at<<<1, 1, 0, st>>>(out, n, nDev);
    ++g_launch_count;
    return;
  }
  k_scan_sums<<<nb, kScanThreads, 0, st>>>(in, n, nDev, scratch);
  ++g_launch_count;
  k_scan_mid<<<1, kScanThreads, 0, st>>>(scratch, nb);
  ++g_launch_count;
  k_scan_apply<<<nb, kScanThreads, 0, st>>>(in, n, nDev, scratch, out);
  ++g_launch_count;
}

// ---- processing order by length (longest first)
__device__ inline int len_bin(const int* __restrict__ off, int i) {
  return kLenBins - 1 - min(off[i + 1] - off[i], kLenBins - 1);
}

__global__ void __launch_bounds__(256) k_len_hist(const int* __restrict__ nDev, const int* __restrict__ off,
                                                  int* __restrict__ hist) {
  __shared__ int sh[kLenBins];
  for (int b = threadIdx.x; b < kLenBins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *nDev) atomicAdd(&sh[len_bin(off, i)], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < kLenBins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

// hist[0, kLenBins) -> exclusive offsets (one CTA of kLenBins threads)
__global__ void __launch_bounds__(kLenBins) k_len_scan(int* __restrict__ hist) {
  __shared__ int sh[kLenBins];
  const int v = hist[threadIdx.x];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int d = 1; d < kLenBins; d <<= 1) {
    const int t = threadIdx.x >= d ? sh[threadIdx.x - d] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  hist[threadIdx.x] = sh[threadIdx.x] - v;
}

// Each block ranks its items per bin in shared memory, then reserves its
// range in each bin with one global atomic per (block, bin).
__global__ void __launch_bounds__(1024) k_len_place(const int* __restrict__ nDev, const int* __restrict__ off,
                                                    int* __restrict__ hist, int* __restrict__ perm) {
  __shared__ int sh[kLenBins];
  for (int b = threadIdx.x; b < kLenBins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int bin = (i < *nDev) ? len_bin(off, i) : -1;
  const int rank = (bin >= 0) ? atomicAdd(&sh[bin], 1) : 0;
  __syncthreads();
  for (int b = threadIdx.x; b < kLenBins; b += blockDim.x)
    if (sh[b]) sh[b] = atomicAdd(&hist[b], sh[b]);
  __syncthreads();
  if (bin >= 0) perm[sh[bin] + rank] = i;
}

void launch_len_order(int n, const int* nDev, const int* off, int* hist, int* perm, cudaStream_t st) {
  if (n <= 0) return;
  cudaMemsetAsync(hist, 0, sizeof(int) * kLenBins, st);
  k_len_hist<<<(n + 255) / 256, 256, 0, st>>>(nDev, off, hist);
  k_len_scan<<<1, kLenBins, 0, st>>>(hist);
  k_len_place<<<(n + 1023) / 1024, 1024, 0, st>>>(nDev, off, hist, perm);
  g_launch_count += 3;
}

// *dst = min(arr[*idx], cap) (a count read off the end of a scan), flagging
// an overflow; optionally also writes the count at base[*dst] (CSR end).
__global__ void k_count_at(const int* __restrict__ arr, const int* __restrict__ idx, int* __restrict__ dst, int cap,
                           int* __restrict__ overflow, const int* __restrict__ arr2, int* __restrict__ dst2, int cap2,
                           int* __restrict__ endBase) {
  int v = arr[*idx];
  if (v > cap) {
    v = cap;
    *overflow = 1;
  }
  *dst = v;
  if (arr2) {
    int v2 = arr2[*idx];
    if (v2 > cap2) {
      v2 = cap2;
      *overflow = 1;
    }
    *dst2 = v2;
    if (endBase) endBase[v] = v2;
  }
}

// first entry of a sorted list that is >= each TF's first sorted hit
__global__ void k_tf_ranges(int nTF, const RowGrid* __restrict__ grid, const int* __restrict__ list,
                            const int* __restrict__ nListDev, int* __restrict__ tfBegin) {
  int tf = blockIdx.x * blockDim.x + threadIdx.x;
  if (tf > nTF) return;
  const int nList = *nListDev;
  int key = (tf == nTF) ? INT_MAX : grid[tf * kRowsPerTF].start;
  int lo = 0, hi = nList;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (list[m] < key) lo = m + 1;
    else hi = m;
  }
  tfBegin[tf] = (tf == nTF) ? nList : lo;
}

// out[i] = first index of the sorted list with list[j] >= keys[i]
__global__ void k_lower_bounds(const int* __restrict__ list, const int* __restrict__ nListDev,
                               const int* __restrict__ keys, int nKeys, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nKeys) return;
  const int nList = *nListDev;
  const int key = keys[i];
  int lo = 0, hi = nList;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (list[m] < key) lo = m + 1;
    else hi = m;
  }
  out[i] = lo;
}

// ------------------------------------------------------------- launchers
void launch_lower_bounds(const int* list, const int* nListDev, const int* keys, int nKeys, int* out,
                         cudaStream_t st) {
  if (nKeys > 0) {
    k_lower_bounds<<<(nKeys + 127) / 128, 128, 0, st>>>(list, nListDev, keys, nKeys, out);
    ++g_launch_count;
  }
}

void launch_neighbours(int nfBlocks, int hitsPerBlock, bool stage, const RowGrid* grid, const int* nfBlockStart,
                       int nRows, const int* cellStart, const int2* syz, const GeomConst* G, int* upRaw, int* dnRaw,
                       unsigned* err, cudaStream_t st, unsigned inject) {
  if (nfBlocks > 0) {
#define O2TPC_NF(B, S) \
  k_neighbours<B, S><<<nfBlocks, B, 0, st>>>(grid, nfBlockStart, nRows, cellStart, syz, G, upRaw, dnRaw, err, inject)
    if (hitsPerBlock == 64) {
      if (stage) O2TPC_NF(64, true);
      else O2TPC_NF(64, false);
    } else if (hitsPerBlock == 256) {
      if (stage) O2TPC_NF(256, true);
      else O2TPC_NF(256, false);
    } else {
      if (stage) O2TPC_NF(128, true);
      else O2TPC_NF(128, false);
    }
#undef O2TPC_NF
    ++g_launch_count;
  }
}

void launch_neighbours_gap(int n, const int* nDev, const RowGrid* grid, int nRows, const int* cellStart,
                           const int2* syz, const GeomConst* G, int* upRaw, int* dnRaw, cudaStream_t st) {
  if (n > 0) {
    k_neighbours_gap<<<(n + 127) / 128, 128, 0, st>>>(nDev, grid, nRows, cellStart, syz, G, upRaw, dnRaw);
    ++g_launch_count;
  }
}

void launch_clean(int n, const int* nDev, const int* upRaw, const int* dnRaw, int* up, int* dn, int* startFlag,
                  cudaStream_t st) {
  if (n > 0) {
    k_clean<<<(n + 255) / 256, 256, 0, st>>>(nDev, upRaw, dnRaw, up, dn, startFlag);
    ++g_launch_count;
  }
}


// ---- ordered compaction with warp ballots
// Flags are taken in tiles of kBallotTile (1024 threads x 4 chunks).  Pass 1
// counts each tile's set flags with one ballot and popcount per warp and
// chunk; the tile counts are scanned; pass 2 writes every flagged index at
// tile offset + earlier chunks + earlier warps (a 32-entry shuffle scan) +
// its rank among the set lanes of its warp (popcount of the lower lanes).
// Only one int per tile is scanned instead of one per flag.
constexpr int kBallotTile = 4096;

__global__ void __launch_bounds__(1024) k_ballot_counts(const int* __restrict__ flag, const int* __restrict__ nDev,
                                                        int* __restrict__ tileCnt) {
  __shared__ int ws[32];
  const int n = *nDev, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = blockIdx.x * kBallotTile + k * 1024 + threadIdx.x;
    c += __popc(__ballot_sync(0xffffffffu, i < n && flag[i] != 0));
  }
  if (lane == 0) ws[w] = c;
  __syncthreads();
  if (w == 0) {
    int v = ws[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) tileCnt[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(1024) k_ballot_compact(const int* __restrict__ flag, const int* __restrict__ nDev,
                                                         const int* __restrict__ tileOff, int* __restrict__ out,
                                                         int cap, int* __restrict__ overflow) {
  __shared__ int ws[32], s_tot;
  const int n = *nDev, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int carry = tileOff[blockIdx.x];
  for (int k = 0; k < 4; ++k) {
    const int i = blockIdx.x * kBallotTile + k * 1024 + threadIdx.x;
    const bool f = i < n && flag[i] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) ws[w] = __popc(m);
    __syncthreads();
    if (w == 0) {  // exclusive scan of the 32 warp counts
      const int v = ws[lane];
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      ws[lane] = x - v;
      if (lane == 31) s_tot = x;
    }
    __syncthreads();
    if (f) {
      const int p = carry + ws[w] + __popc(m & ((1u << lane) - 1u));
      if (p < cap) out[p] = i;
      else *overflow = 1;
    }
    carry += s_tot;
    __syncthreads();
  }
}

// *dst = min(total, cap) with total = tileOff[number of tiles of *nDev]
__global__ void k_ballot_total(const int* __restrict__ tileOff, const int* __restrict__ nDev, int* __restrict__ dst,
                               int cap, int* __restrict__ overflow) {
  int v = tileOff[(*nDev + kBallotTile - 1) / kBallotTile];
  if (v > cap) {
    v = cap;
    *overflow = 1;
  }
  *dst = v;
}

int ballot_tiles(long long n) { return (int)((n + kBallotTile - 1) / kBallotTile); }

void launch_ballot_count(int n, const int* nDev, const int* flag, int* tileCnt, int* tileOff, int* count, int cap,
                         int* overflow, int* scratch, cudaStream_t st) {
  const int nt = ballot_tiles(n);
  if (nt > 0) {
    k_ballot_counts<<<nt, 1024, 0, st>>>(flag, nDev, tileCnt);
    ++g_launch_count;
  }
  // tiles past *nDev count zero; the scan runs over all nt
  scan_exclusive(tileCnt, tileOff, nt, nullptr, scratch, st);
  k_ballot_total<<<1, 1, 0, st>>>(tileOff, nDev, count, cap, overflow);
  ++g_launch_count;
}

void launch_ballot_compact(int n, const int* nDev, const int* flag, const int* tileOff, int* out, int cap,
                           int* overflow, cudaStream_t st) {
  const int nt = ballot_tiles(n);
  if (nt > 0) {
    k_ballot_compact<<<nt, 1024, 0, st>>>(flag, nDev, tileOff, out, cap, overflow);
    ++g_launch_count;
  }
}

__global__ void k_iota(int* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = i;
}

__global__ void k_stream_tail() {}

void launch_stream_tail(cudaStream_t st) {
  k_stream_tail<<<1, 32, 0, st>>>();
  ++g_launch_count;
}

void launch_iota(int* out, int n, cudaStream_t st) {
  if (n > 0) {
    k_iota<<<(n + 255) / 256, 256, 0, st>>>(out, n);
    ++g_launch_count;
  }
}

void launch_count_at(const int* arr, const int* idx, int* dst, int cap, int* overflow, cudaStream_t st,
                     const int* arr2, int* dst2, int cap2, int* endBase) {
  k_count_at<<<1, 1, 0, st>>>(arr, idx, dst, cap, overflow, arr2, dst2, cap2, endBase);
  ++g_launch_count;
}

void launch_tf_ranges(int nTF, const RowGrid* grid, const int* list, const int* nListDev, int* tfBegin,
                      cudaStream_t st) {
  k_tf_ranges<<<(nTF + 1 + 63) / 64, 64, 0, st>>>(nTF, grid, list, nListDev, tfBegin);
  ++g_launch_count;
}

}  // namespace o2tpc
