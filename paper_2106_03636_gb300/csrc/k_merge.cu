// k_merge.cu - sector-to-sector merger, chain building and final refit.
//
// Border tracks: a sector track whose outer end lies within 5 cm of a sector
// edge (|y| >= x tan 10 deg - 5) may continue in the neighbouring sector of
// the same side as a track whose inner end lies at the shared edge.  For
// each such pair (prefilter: endpoint drift coordinates within 20 cm) the
// outer state is rotated into the neighbour's frame, transported to the
// neighbour's inner x, and compared on all five parameters with the summed
// covariance (chi2 <= 30).  Per directed sector edge the pairs are taken
// greedily in ascending (chi2, a, b), each track end at most once; linked
// sector tracks form chains (a closed loop is cut at its smallest id).  The
// final refit runs inward over each chain's clusters, rotating at sector
// boundaries, in FP32; a track whose FP32 covariance stops being positive
// definite after an update is redone with an FP64 covariance and counted.
#include <algorithm>

#include "o2tpc_kernels.cuh"

namespace o2tpc {

__device__ inline int nb_sector(int s, int d) { return (s / 18) * 18 + (s % 18 + d + 18) % 18; }

// Keys: inner end of a border track -> B-list key (tf*36 + sector)*2 + (dir>0);
// outer end -> the edge key of the same form for its own sector.
__global__ void k_merge_keys(SectorTrackBufs sb, const GeomConst* __restrict__ G, MergeBufs mb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mb.cnt->nSt) return;
  const float tn = G->tan10;
  const float* so = sb.out + (size_t)i * 21;
  const float* si = sb.in + (size_t)i * 21;
  const int base = (sb.tf[i] * kNSec + sb.sector[i]) * 2;
  int ko = -1, ki = -1;
  if (fabsf(so[1]) >= so[0] * tn - kEdgeBand) ko = base + (so[1] > 0.f ? 1 : 0);
  if (fabsf(si[1]) >= si[0] * tn - kEdgeBand) {
    ki = base + (si[1] > 0.f ? 1 : 0);
    atomicAdd(&mb.listCnt[ki], 1);
  }
  mb.keyOut[i] = ko;
  mb.keyIn[i] = ki;
  mb.next[i] = -1;
  mb.prev[i] = -1;
  mb.reached[i] = 0;
}

// Drift coordinate of a state in integer units (origin zref); the merge
// window search only needs it to a few units.
__device__ inline int zeta_units(int zref, float zrel, float zunit) {
  return zref + (int)lrintf(fminf(fmaxf(zrel / zunit, -1.0e9f), 1.0e9f));
}

__global__ void k_merge_list_fill(SectorTrackBufs sb, const GeomConst* __restrict__ G, MergeBufs mb,
                                  int* __restrict__ cursor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mb.cnt->nSt) return;
  const int k = mb.keyIn[i];
  if (k < 0) return;
  const int slot = mb.listStart[k] + atomicAdd(&cursor[k], 1);
  mb.listItems[slot] = i;
  mb.listKey[slot] = zeta_units(sb.zref[i], sb.in[(size_t)i * 21 + 2], G->zunit);
}

constexpr int kListSmem = 8192;

// Bitonic sort by one CTA of buf[0, n2) (n2 a power of two, padding already
// holding keys that sort last); buf may live in shared or global memory.
template <typename T, typename Less>
__device__ void cta_bitonic(T* buf, int n2, Less less) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const T x = buf[i], y = buf[l];
          if (((i & k) == 0) ? less(y, x) : less(x, y)) {
            buf[i] = y;
            buf[l] = x;
          }
        }
      }
      __syncthreads();
    }
}

struct KeyLess {
  __device__ bool operator()(const int2& x, const int2& y) const { return x.x < y.x || (x.x == y.x && x.y < y.y); }
};

// The same bitonic network for n2 > kListSmem items in global memory g: the
// stages up to kListSmem, and at every later stage the steps of distance <
// kListSmem, run on one kListSmem chunk at a time staged in shared memory
// sm; only the steps of distance >= kListSmem make passes over g.  The
// direction of a compare-exchange is taken from the global index.
__device__ void list_bitonic_big(int2* g, int n2, int2* sm) {
  constexpr int S = kListSmem;
  const KeyLess less;
  auto cx = [&](int2* buf, int i, int l, int gi, int k) {
    const int2 x = buf[i], y = buf[l];
    if (((gi & k) == 0) ? less(y, x) : less(x, y)) {
      buf[i] = y;
      buf[l] = x;
    }
  };
  // stages k <= S: each chunk sorted on its own (its direction from the chunk's index)
  for (int c = 0; c < n2; c += S) {
    for (int i = threadIdx.x; i < S; i += blockDim.x) sm[i] = g[c + i];
    __syncthreads();
    for (int k = 2; k <= S; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) cx(sm, i, l, c + i, k);
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < S; i += blockDim.x) g[c + i] = sm[i];
    __syncthreads();
  }
  for (int k = 2 * S; k <= n2; k <<= 1) {
    for (int j = k >> 1; j >= S; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) cx(g, i, l, i, k);
      }
      __syncthreads();
    }
    for (int c = 0; c < n2; c += S) {
      for (int i = threadIdx.x; i < S; i += blockDim.x) sm[i] = g[c + i];
      __syncthreads();
      for (int j = S >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) cx(sm, i, l, c + i, k);
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < S; i += blockDim.x) g[c + i] = sm[i];
      __syncthreads();
    }
  }
}

// One CTA per B list: sort it by drift coordinate (bitonic, in shared memory
// up to kListSmem items, else in the global scratch at 2 * listStart, which
// has room for the padded power of two, with the short-distance steps staged
// through shared memory chunk by chunk).
__global__ void __launch_bounds__(512) k_merge_list_sort(MergeBufs mb, int2* __restrict__ scratch) {
  __shared__ int2 sk[kListSmem];
  const int b = mb.listStart[blockIdx.x], n = mb.listStart[blockIdx.x + 1] - b;
  if (n <= 1) return;
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  int2* buf = (n2 <= kListSmem) ? sk : scratch + 2 * (size_t)b;
  for (int i = threadIdx.x; i < n2; i += blockDim.x)
    buf[i] = (i < n) ? make_int2(mb.listKey[b + i], mb.listItems[b + i]) : make_int2(INT_MAX, INT_MAX);
  __syncthreads();
  if (n2 <= kListSmem) cta_bitonic(buf, n2, KeyLess());
  else list_bitonic_big(buf, n2, sk);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mb.listKey[b + i] = buf[i].x;
    mb.listItems[b + i] = buf[i].y;
  }
}

// Cholesky chi2 = d^T M^-1 d of a symmetric 5x5 (lower triangle); false if
// M is not positive definite.
__device__ inline bool chi2_5(const float* d, const float* M, float& out) {
  float L[15];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float s = M[ix(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= L[ix(i, k)] * L[ix(j, k)];
      if (i == j) {
        if (!(s > 0.f)) return false;
        L[ix(i, i)] = sqrtf(s);
      } else {
        L[ix(i, j)] = s / L[ix(j, j)];
      }
    }
  float v[5], c = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float s = d[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[ix(i, k)] * v[k];
    v[i] = s / L[ix(i, i)];
    c += v[i] * v[i];
  }
  out = c;
  return true;
}

// One thread per outer border end A: all B candidates of the neighbour edge.
__global__ void __launch_bounds__(128) k_merge_pairs(SectorTrackBufs sb, const GeomConst* __restrict__ G,
                                                     MergeBufs mb, unsigned* __restrict__ err) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= mb.cnt->nSt) return;
  const int ko = mb.keyOut[a];
  if (ko < 0) return;
  const int d = (ko & 1) ? 1 : -1;
  const int s2 = nb_sector(sb.sector[a], d);
  const int kb = (sb.tf[a] * kNSec + s2) * 2 + (d > 0 ? 0 : 1);
  int b0 = mb.listStart[kb], b1 = mb.listStart[kb + 1];
  if (b0 == b1) return;
  const float zunit = G->zunit, bzc = G->bzc;
  KState<float> A;
  {
    const float* so = sb.out + (size_t)a * 21;
    A.x = so[0];
#pragma unroll
    for (int q = 0; q < 5; ++q) A.p[q] = so[1 + q];
#pragma unroll
    for (int q = 0; q < 15; ++q) A.C[q] = so[6 + q];
  }
  const int zra = sb.zref[a];
  KState<float> Ar = A;
  const bool rotOk = kf_rotate<float>(Ar, G->rot_cos, d * G->rot_sin, bzc) == 0;
  if (!rotOk) return;
  {
    // sorted list: only the drift-coordinate window (a superset of the
    // prefilter below, 4 units of margin for rounding)
    const int za = zeta_units(zra, A.p[1], zunit);
    const int w = (int)ceilf(kMergeDZeta / zunit) + 4;
    int lo = b0, hi = b1;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (mb.listKey[m] < za - w) lo = m + 1;
      else hi = m;
    }
    const int first = lo;
    lo = first;
    hi = b1;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (mb.listKey[m] <= za + w) lo = m + 1;
      else hi = m;
    }
    b0 = first;
    b1 = lo;
  }
  for (int q = b0; q < b1; ++q) {
    const int b = mb.listItems[q];
    const float* B = sb.in + (size_t)b * 21;
    const float dzr = (float)(zra - sb.zref[b]) * zunit;
    if (fabsf(dzr + A.p[1] - B[2]) > kMergeDZeta) continue;
    KState<float> t = Ar;
    if (kf_prop<float>(t, B[0], bzc) != 0) continue;
    float dv[5], cs[15];
#pragma unroll
    for (int k = 0; k < 5; ++k) dv[k] = t.p[k] - B[1 + k];
    dv[1] += dzr;
#pragma unroll
    for (int k = 0; k < 15; ++k) cs[k] = t.C[k] + B[6 + k];
    float c2;
    if (!chi2_5(dv, cs, c2)) continue;
    if (!(c2 <= kChi2Merge)) continue;
    const int slot = atomicAdd(mb.pairCount, 1);
    if (slot < mb.pairCap) mb.pairs[slot] = make_float4(c2, __int_as_float(a), __int_as_float(b), __int_as_float(ko));
    else atomicOr(err, kErrOverflow);
  }
}


__global__ void k_pair_hist(MergeBufs mb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = min(*mb.pairCount, mb.pairCap);
  if (i >= n) return;
  atomicAdd(&mb.edgeCnt[__float_as_int(mb.pairs[i].w)], 1);
}

__global__ void k_pair_group(MergeBufs mb, int* __restrict__ cursor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = min(*mb.pairCount, mb.pairCap);
  if (i >= n) return;
  const float4 p = mb.pairs[i];
  const int e = __float_as_int(p.w);
  mb.pairsSorted[mb.edgeStart[e] + atomicAdd(&cursor[e], 1)] = p;
}

// One CTA per directed edge: the greedy matching in ascending (chi2, a, b),
// each track end used once, computed without ordering the pairs.  A pair
// that is the smallest among the still-free pairs at both of its ends would
// be taken by the sequential greedy pass as well (every smaller pair at its
// ends lost an end to a pair taken before it), so taking all such pairs at
// once, and repeating on the pairs whose ends are both still free, yields
// exactly the greedy result; the smallest free pair of the edge qualifies in
// every round, so the rounds end.  The minima use 64-bit keys: for pairs
// sharing end a, (chi2 bits, b); for pairs sharing b, (chi2 bits, a)
// (chi2 >= 0, so its float bits order like the value).  minA / minB are
// indexed by track; every track end belongs to a single edge.
__global__ void __launch_bounds__(512) k_merge_select(MergeBufs mb, unsigned long long* __restrict__ minA,
                                                      unsigned long long* __restrict__ minB) {
  const int e = blockIdx.x;
  const int b0 = mb.edgeStart[e], b1 = mb.edgeStart[e + 1];
  if (b0 == b1) return;
  const float4* P = mb.pairsSorted;
  for (int round = 0; round <= b1 - b0; ++round) {
    int alive = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      const float4 p = P[i];
      const int a = __float_as_int(p.y), b = __float_as_int(p.z);
      if (mb.next[a] < 0 && mb.prev[b] < 0) {
        minA[a] = ~0ull;
        minB[b] = ~0ull;
        alive = 1;
      }
    }
    if (!__syncthreads_or(alive)) break;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      const float4 p = P[i];
      const int a = __float_as_int(p.y), b = __float_as_int(p.z);
      if (mb.next[a] < 0 && mb.prev[b] < 0) {
        const unsigned long long c = (unsigned long long)(unsigned)__float_as_int(p.x) << 32;
        atomicMin(&minA[a], c | (unsigned)b);
        atomicMin(&minB[b], c | (unsigned)a);
      }
    }
    __syncthreads();
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      const float4 p = P[i];
      const int a = __float_as_int(p.y), b = __float_as_int(p.z);
      if (mb.next[a] < 0 && mb.prev[b] < 0) {
        const unsigned long long c = (unsigned long long)(unsigned)__float_as_int(p.x) << 32;
        if (minA[a] == (c | (unsigned)b) && minB[b] == (c | (unsigned)a)) {
          mb.next[a] = b;
          mb.prev[b] = a;
        }
      }
    }
    __syncthreads();
  }
}

// Chains: mark every track reachable from a head (prev < 0).
__global__ void k_chain_reach(MergeBufs mb) {
  const int nSt = mb.cnt->nSt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nSt || mb.prev[i] >= 0) return;
  int guard = 0;
  for (int c = i; c >= 0 && guard <= nSt; c = mb.next[c], ++guard) mb.reached[c] = 1;
}

// Cut every closed loop of links at its smallest id.  A track not reached
// from any head lies on a loop; walking the loop (links unchanged in this
// kernel) finds whether it is the loop's smallest member, which marks itself.
// The next kernel cuts the link into every marked track, so each loop is cut
// exactly once, whatever the thread order.
__global__ void k_chain_loops(MergeBufs mb) {
  const int nSt = mb.cnt->nSt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nSt || mb.reached[i]) return;
  int mn = i, guard = 0;
  for (int c = mb.next[i]; c >= 0 && c != i && guard < nSt; c = mb.next[c], ++guard) mn = min(mn, c);
  if (mn == i) mb.reached[i] = 2;
}

__global__ void k_chain_loops_fix(MergeBufs mb) {
  const int nSt = mb.cnt->nSt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nSt || mb.reached[i] != 2) return;
  const int p = mb.prev[i];
  if (p >= 0) mb.next[p] = -1;
  mb.prev[i] = -1;
}

__global__ void k_head_flags(MergeBufs mb, int* __restrict__ headFlag) {
  const int nSt = mb.cnt->nSt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nSt) headFlag[i] = mb.prev[i] < 0;
}


__global__ void k_chain_counts(const int* __restrict__ nHeadsDev, const int* __restrict__ heads, SectorTrackBufs sb,
                               MergeBufs mb,
                               int* __restrict__ trkNcl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nHeadsDev) return;
  int n = 0, nseg = 0;
  for (int c = heads[t]; c >= 0 && nseg < kMaxChain; c = mb.next[c], ++nseg) n += sb.off[c + 1] - sb.off[c];
  trkNcl[t] = n;
}

// Inward refit over a chain of sector tracks from its tail (the last of at
// most kMaxChain segments) back to its head through the prev links, hits of
// each segment descending in rows, in precision T.  y is kept relative to
// the origin yref (integer units), moved in whole centimetres to each hit
// before its update, and zeta relative to the hit itself (recentre_z; zeta
// is put back relative to zref at the end); at a sector boundary the state is
// made absolute,
// rotated, and re-referenced to the next hit.  Steps between pad rows come
// from the row pitch; the first step after a rotation (x off the rows) from
// the positions.  Returns flags bits 2 (stopped at a
// boundary) and 8 (FP32 covariance lost positive definiteness); yref of the
// final state in *yrefOut.
template <typename T>
__device__ int refit_chain(int head, int tail, const SectorTrackBufs& sb, const int* __restrict__ prev,
                           const int2* __restrict__ syz, const GeomConst* __restrict__ G, int zref, KState<T>& t,
                           T& chi2, int& used, int& frame, int* yrefOut) {
  const T zunit = sizeof(T) == 8 ? (T)G->zunit_d : (T)G->zunit;
  const T bzc = sizeof(T) == 8 ? (T)G->bzc_d : (T)G->bzc;
  const T rc = sizeof(T) == 8 ? (T)G->rot_cos_d : (T)G->rot_cos;
  const T rs = sizeof(T) == 8 ? (T)G->rot_sin_d : (T)G->rot_sin;
  const T yunit = T(1) / T(160);
  frame = sb.sector[tail];
  const int hl = sb.off[tail + 1] - 1;
  const float* so = sb.out + (size_t)tail * 21;
  const int2 pl = sb.yz[hl];
  int yref = pl.x;
  const T xl = sizeof(T) == 8 ? (T)G->rowx_d[sb.rows[hl]] : (T)G->rowx[sb.rows[hl]];
  kf_reset<T>(t, xl, T(0), T(0), (T)so[3], (T)so[4], (T)so[5]);  // at the last hit: the origins
  kf_meas_cov<T>(t, G->angErr);
  int srow = sb.rows[hl];  // row of the state, -1 after a rotation
  int zcur = pl.y;         // drift origin of the fit, moved to each hit
  chi2 = T(0);
  used = 1;
  int flags = 0;
  bool first = true;
  for (int sg = tail;; sg = prev[sg]) {
    const int sec = sb.sector[sg];
    for (int i = sb.off[sg + 1] - 1; i >= sb.off[sg]; --i) {
      if (first) { first = false; continue; }
      const int2 p = sb.yz[i];
      if (sec != frame) {
        const int dd = ((sec % 18) - (frame % 18) + 18) % 18;
        const T sgn = (dd == 1) ? T(1) : T(-1);
        t.p[0] += (T)yref * yunit;
        if (kf_rotate<T>(t, rc, sgn * rs, bzc) != 0) {
          t.p[0] -= (T)yref * yunit;
          t.p[1] += (T)(zcur - zref) * zunit;
          *yrefOut = yref;
          return flags | 4;
        }
        yref = p.x;
        t.p[0] -= (T)yref * yunit;
        frame = sec;
        srow = -1;
      }
      const int ri = sb.rows[i];
      if constexpr (sizeof(T) == 8) {  // FP64 fallback: single-precision geometry, double covariance
        const float dx = srow >= 0 ? (float)(ri - srow) * G->pitch : (float)(G->rowx_d[ri] - (double)t.x);
        if (kf_prop_dx_cov64(t, G->rowx_d[ri], dx, G->bzc) != 0) continue;
      } else if (srow >= 0) {
        if (kf_prop_row<T>(t, srow, ri, G, bzc) != 0) continue;
      } else {
        if (kf_prop<T>(t, (T)G->rowx[ri], bzc) != 0) continue;
      }
      srow = ri;
      recentre_y<T>(t.p[0], yref, p.x);
      recentre_z<T>(t.p[1], zcur, p.y, zunit);
      T c2;
      if (kf_update<T>(t, (T)(p.x - yref) * yunit, T(0), &c2, G->angErr) != 0) continue;
      chi2 += c2;
      ++used;
      if (!kf_cov_ok<T>(t.C)) flags |= 8;
    }
    if (sg == head) break;
  }
  t.p[1] += (T)(zcur - zref) * zunit;  // zeta back to the track's origin
  *yrefOut = yref;
  return flags;
}

// Output row t of a track: state at the innermost cluster in the frame of
// its sector, tan(lambda) = dz/ds = -side * dzeta/ds.
template <typename T>
__device__ void write_track(int t, const KState<T>& s, int yref, T chi2, int used, int frame, int flags, int zref,
                            const GeomConst* __restrict__ G, OutBufs& ob) {
  float par[5], cov[15];
#pragma unroll
  for (int k = 0; k < 5; ++k) par[k] = (float)s.p[k];
  par[0] = (float)((double)s.p[0] + (double)yref / 160.0);
#pragma unroll
  for (int k = 0; k < 15; ++k) cov[k] = (float)s.C[k];
  const float sg = (frame < 18) ? -1.f : 1.f;
  par[3] *= sg;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (k != 3) cov[ix(3, k)] *= sg;
  ob.x[t] = (float)s.x;
  ob.alpha[t] = G->sec_alpha[frame % 18];
#pragma unroll
  for (int k = 0; k < 5; ++k) ob.par[(size_t)t * 5 + k] = par[k];
#pragma unroll
  for (int k = 0; k < 15; ++k) ob.cov[(size_t)t * 15 + k] = cov[k];
  ob.chi2[t] = (float)chi2;
  ob.ndf[t] = 2 * used - 5;
  ob.sector[t] = (uint8_t)frame;
  ob.flags[t] = (uint8_t)flags;
  ob.zref[t] = zref;
}

// Tail of a chain: the last of at most kMaxChain segments from its head.
__device__ inline int chain_tail(int head, const int* __restrict__ next, int* nseg) {
  int tail = head, n = 1;
  for (int c = next[head]; c >= 0 && n < kMaxChain; c = next[c], ++n) tail = c;
  *nseg = n;
  return tail;
}

// K11: final refit in FP32, one thread per track; cluster list in chain
// order, ascending rows inside each segment, as indices into the TF's
// submitted order.  A track whose FP32 covariance stops being positive
// definite (or every track with forceFp64) is queued for k_final_refit64.
__global__ void __launch_bounds__(128) k_final_refit(const int* __restrict__ nHeadsDev, const int* __restrict__ heads,
                                                     SectorTrackBufs sb,
                                                     MergeBufs mb, const int2* __restrict__ syz,
                                                     const int* __restrict__ sorig, const TFDesc* __restrict__ tfs,
                                                     const GeomConst* __restrict__ G, int forceFp64, OutBufs ob) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nHeadsDev) return;
  const int head = heads[t];
  int nseg;
  const int tail = chain_tail(head, mb.next, &nseg);
  const int tf = sb.tf[head];
  const int inBase = tfs[tf].inBase;
  int o = ob.off[t];
  for (int c = head, j = 0; j < nseg; c = mb.next[c], ++j)
    for (int i = sb.off[c]; i < sb.off[c + 1]; ++i) ob.cl[o++] = sb.orig[i] - inBase;
  const int zref = sb.yz[sb.off[head]].y;
  {
    // the drift coordinate is linear along the helix: its extremes over the
    // track are those of the two end clusters
    const int hl = sb.off[tail + 1] - 1;
    const int zl = sb.yz[hl].y;
    ob.ends[t] = make_int4(min(zref, zl), max(zref, zl), zref, zl);
    ob.endsR[t] = make_int2(sb.rows[sb.off[head]] | (sb.rows[hl] << 8) | (sb.sector[head] << 16) |
                                (sb.sector[tail] << 24),
                            tf);
  }
  KState<float> sf;
  float c2f;
  int used, frame, yref;
  const int fl = refit_chain<float>(head, tail, sb, mb.prev, syz, G, zref, sf, c2f, used, frame, &yref);
  if ((fl & 8) || forceFp64) {
    ob.fallback[atomicAdd(ob.nFallback, 1)] = t;
    return;
  }
  write_track<float>(t, sf, yref, c2f, used, frame, (nseg > 1 ? 2 : 0) | (fl & 4), zref, G, ob);
}

// K11b: the queued tracks again with an FP64 covariance (flag bit 1): the
// state and its covariance in double, each transport step's geometry in
// single precision (kf_prop_dx_cov64).
__global__ void __launch_bounds__(128) k_final_refit64(const int* __restrict__ heads, SectorTrackBufs sb, MergeBufs mb,
                                                       const int2* __restrict__ syz, const GeomConst* __restrict__ G,
                                                       OutBufs ob) {
  const int nf = *ob.nFallback;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x) {
    const int t = ob.fallback[q];
    const int head = heads[t];
    int nseg;
    const int tail = chain_tail(head, mb.next, &nseg);
    const int zref = sb.yz[sb.off[head]].y;
    KState<double> sd;
    double c2d;
    int used, frame, yref;
    const int fl = refit_chain<double>(head, tail, sb, mb.prev, syz, G, zref, sd, c2d, used, frame, &yref);
    write_track<double>(t, sd, yref, c2d, used, frame, 1 | (nseg > 1 ? 2 : 0) | (fl & 4), zref, G, ob);
  }
}

// ------------------------------------------------------------- launchers
// nSt, nKeys, nPairs, nHeads below size the grids (exact or capacities); the
// kernels read the sizes from mb.cnt / nHeadsDev.
void launch_merge_keys(int nSt, const SectorTrackBufs sb, const GeomConst* G, MergeBufs mb, int nKeys, int* scratch,
                       cudaStream_t st) {
  cudaMemsetAsync(mb.listCnt, 0, sizeof(int) * (nKeys + 1), st);
  if (nSt > 0) {
    k_merge_keys<<<(nSt + 255) / 256, 256, 0, st>>>(sb, G, mb);
    ++g_launch_count;
  }
  scan_exclusive(mb.listCnt, mb.listStart, nKeys, &mb.cnt->nKeys, scratch, st);
  cudaMemsetAsync(mb.listCnt, 0, sizeof(int) * (nKeys + 1), st);
  if (nSt > 0) {
    k_merge_list_fill<<<(nSt + 255) / 256, 256, 0, st>>>(sb, G, mb, mb.listCnt);
    ++g_launch_count;
  }
  if (nKeys > 0) {
    k_merge_list_sort<<<nKeys, 512, 0, st>>>(mb, reinterpret_cast<int2*>(mb.sortScratch));
    ++g_launch_count;
  }
}

void launch_list_sort(int nKeys, MergeBufs mb, cudaStream_t st) {
  if (nKeys > 0) {
    k_merge_list_sort<<<nKeys, 512, 0, st>>>(mb, reinterpret_cast<int2*>(mb.sortScratch));
    ++g_launch_count;
  }
}

void launch_merge_pairs(int nSt, const SectorTrackBufs sb, const GeomConst* G, MergeBufs mb, unsigned* err,
                        cudaStream_t st) {
  cudaMemsetAsync(mb.pairCount, 0, sizeof(int), st);
  if (nSt > 0) {
    k_merge_pairs<<<(nSt + 127) / 128, 128, 0, st>>>(sb, G, mb, err);
    ++g_launch_count;
  }
}

void launch_merge_select(int nPairs, int nKeys, MergeBufs mb, int* scratch, cudaStream_t st) {
  cudaMemsetAsync(mb.edgeCnt, 0, sizeof(int) * (nKeys + 1), st);
  if (nPairs > 0) {
    k_pair_hist<<<(nPairs + 255) / 256, 256, 0, st>>>(mb);
    ++g_launch_count;
  }
  scan_exclusive(mb.edgeCnt, mb.edgeStart, nKeys, &mb.cnt->nKeys, scratch, st);
  cudaMemsetAsync(mb.edgeCnt, 0, sizeof(int) * (nKeys + 1), st);
  if (nPairs > 0) {
    k_pair_group<<<(nPairs + 255) / 256, 256, 0, st>>>(mb, mb.edgeCnt);
    ++g_launch_count;
  }
  if (nKeys > 0) {
    auto* minA = reinterpret_cast<unsigned long long*>(mb.sortScratch);
    k_merge_select<<<nKeys, 512, 0, st>>>(mb, minA, minA + mb.nSt);
    ++g_launch_count;
  }
}

void launch_chains(int nSt, MergeBufs mb, int* headFlag, cudaStream_t st) {
  if (nSt > 0) {
    k_chain_reach<<<(nSt + 255) / 256, 256, 0, st>>>(mb);
    k_chain_loops<<<(nSt + 255) / 256, 256, 0, st>>>(mb);
    k_chain_loops_fix<<<(nSt + 255) / 256, 256, 0, st>>>(mb);
    k_head_flags<<<(nSt + 255) / 256, 256, 0, st>>>(mb, headFlag);
    g_launch_count += 4;
  }
}

void launch_chain_counts(int nHeads, const int* nHeadsDev, const int* heads, const SectorTrackBufs sb, MergeBufs mb,
                         int* trkNcl, cudaStream_t st) {
  if (nHeads > 0) {
    k_chain_counts<<<(nHeads + 255) / 256, 256, 0, st>>>(nHeadsDev, heads, sb, mb, trkNcl);
    ++g_launch_count;
  }
}

void launch_final_refit(int nHeads, const int* nHeadsDev, const int* heads, const SectorTrackBufs sb, MergeBufs mb,
                        const int2* syz, const int* sorig, const TFDesc* tfs, const GeomConst* G, int forceFp64,
                        OutBufs ob, cudaStream_t st) {
  if (nHeads > 0) {
    k_final_refit<<<(nHeads + 127) / 128, 128, 0, st>>>(nHeadsDev, heads, sb, mb, syz, sorig, tfs, G, forceFp64,
                                                         ob);
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    k_final_refit64<<<std::min((nHeads + 127) / 128, sms * 4), 128, 0, st>>>(heads, sb, mb, syz, G, ob);
    g_launch_count += 2;
  }
}

}  // namespace o2tpc
