// Continuous-readout completion (Sec. 2): collision time t0 of every final
// track, links between the two halves of a track that crosses the central
// membrane, and assignment of tracks to the TF's interaction times.
//
// With continuous readout a cluster's drift coordinate is
// zeta = v_d (t0 + t_drift) = v_d t0 + 250 cm - |z|, so the clusters of one
// track fix t0 only up to the z of its vertex.  The paper leaves the method
// open; the rules below are this implementation's reading:
//  * bounds: 0 <= |z| <= 250 cm for every cluster gives
//    zeta_max - 250 <= v_d t0 <= zeta_min, where zeta is linear along the
//    helix, so its extremes are taken at the track's two end clusters;
//  * vertex t0: the track followed back to its closest approach to the beam
//    axis in the transverse plane, where z_vertex = 0 is assumed; the result
//    is clamped into the bounds; its error adds a 5 cm beam-spot length;
//  * membrane link: an inner piece running towards z = 0 that ends before the
//    last row, and an outer piece on the other side (same sector angle or a
//    neighbouring one) starting 1-10 rows further out with a drift coordinate
//    within 384 units, are one particle when y, sin(phi), tan(lambda), q/pT
//    agree (chi2 <= 25 on the four) at the outer piece's first cluster and
//    the membrane (the mean of the two drift coordinates there, since z is
//    continuous across it) lies no more than 1 cm below any of their
//    clusters.  Each piece takes one partner, greedy in (chi2, inner, outer),
//    and both get t0 = (zeta_membrane - 250) / v_d and the intersection of
//    their bounds;
//  * assignment: among the interaction times of the TF compatible with the
//    bounds widened by 0.3 us, the one nearest to t0 (ties: the earlier).
//
// Data flow per batch, after the final refit (which leaves each track's
// first/last cluster, drift range and TF in ob.ends / ob.endsR):
//   k_cont_keys       classify the pieces; outer pieces counted per (TF, sector)
//   scan, k_cont_fill outer pieces listed per (TF, sector), keyed by first zeta
//   list sort         (the merger's per-list bitonic sort)
//   k_cont_pairs      one thread per inner piece: candidate pairs
//   pair selection    (the merger's exact parallel greedy, one CTA per TF)
//   k_cont_t0         t0, error, bounds, partner and collision per track
// The merger's buffers are free by then and are reused (sizes: tracks <=
// sector tracks).
#include "o2tpc_internal.cuh"
#include "o2tpc_kernels.cuh"

namespace o2tpc {

namespace {

constexpr float kSigmaZv = 5.0f;      // beam-spot length, cm
constexpr int kMemRowGap = 10;        // outer piece starts 1..10 rows further out
constexpr int kMemDZetaUnits = 384;   // first-zeta window of the outer piece
constexpr float kChi2Mem = 25.0f;     // on 4 parameters
constexpr float kMemZTol = 1.0f;      // cm
constexpr double kT0Slack = 0.3;      // us, on the bounds when assigning

__device__ inline int side_of(int sector) { return sector < 18 ? 1 : -1; }

// Output state of track t in the tracker's convention (p[3] = dzeta/ds).
__device__ inline void load_track(const OutBufs& ob, int t, KState<float>& s) {
  s.x = ob.x[t];
#pragma unroll
  for (int k = 0; k < 5; ++k) s.p[k] = ob.par[(size_t)t * 5 + k];
#pragma unroll
  for (int k = 0; k < 15; ++k) s.C[k] = ob.cov[(size_t)t * 15 + k];
  const float sg = ob.sector[t] < 18 ? -1.f : 1.f;
  s.p[3] *= sg;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (k != 3) s.C[ix(3, k)] *= sg;
}

// Cholesky chi2 = d^T M^-1 d of a symmetric 4x4 (lower triangle, ix order).
__device__ inline bool chi2_4(const float* d, const float* M, float& out) {
  float L[10];
#pragma unroll
  for (int i = 0; i < 4; ++i)
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
  float v[4], c = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float s = d[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[ix(i, k)] * v[k];
    v[i] = s / L[ix(i, i)];
    c += v[i] * v[i];
  }
  out = c;
  return true;
}

struct Ends {
  int zmin, zmax, zin, zout;
  int rin, rout, sin, sout, tf;
};

__device__ inline Ends load_ends(const OutBufs& ob, int t) {
  const int4 z = ob.ends[t];
  const int2 r = ob.endsR[t];
  Ends e;
  e.zmin = z.x;
  e.zmax = z.y;
  e.zin = z.z;
  e.zout = z.w;
  e.rin = r.x & 0xff;
  e.rout = (r.x >> 8) & 0xff;
  e.sin = (r.x >> 16) & 0xff;
  e.sout = (r.x >> 24) & 0xff;
  e.tf = r.y;
  return e;
}

// An inner piece: single frame at its first cluster, runs towards z = 0,
// ends before the last row.
__device__ inline bool inner_piece(const OutBufs& ob, int t, const Ends& e) {
  if ((ob.flags[t] & 4) || ob.sector[t] != e.sin || e.rout > kNRow - 2) return false;
  return side_of(e.sout) * ob.par[(size_t)t * 5 + 3] < 0.f;
}

// An outer piece: starts after the first row and runs away from z = 0.
__device__ inline bool outer_piece(const OutBufs& ob, int t, const Ends& e) {
  if ((ob.flags[t] & 4) || ob.sector[t] != e.sin || e.rin < 1) return false;
  return side_of(e.sin) * ob.par[(size_t)t * 5 + 3] > 0.f;
}

// Inner piece a against outer piece b: true with chi2, the membrane drift
// coordinate (cm, relative to a's zeta_ref) and its variance when they are
// one particle.  The t0 kernel calls it again on a pair already taken with
// cuts = false: the same operations then give the membrane coordinate even
// if a cut compared differently there by a rounding (not inlined: both
// kernels run the same machine code).
__device__ __noinline__ bool membrane_match(const OutBufs& ob, const GeomConst* __restrict__ G, int a, const Ends& ea,
                                      int b, const Ends& eb, bool cuts, float& chi2, float& zmRel, float& zmVar) {
  const int gap = eb.rin - ea.rout;
  if (cuts && (gap < 1 || gap > kMemRowGap)) return false;
  if (cuts && abs(eb.zin - ea.zout) > kMemDZetaUnits) return false;
  const int jrot = (((eb.sin % 18) - (ea.sin % 18)) % 18 + 27) % 18 - 9;
  if (cuts && (jrot < -2 || jrot > 2)) return false;
  KState<float> t;
  load_track(ob, a, t);
  const float sga = ob.sector[a] < 18 ? -1.f : 1.f;
  for (int r = 0; r < (jrot < 0 ? -jrot : jrot); ++r)
    if (kf_rotate<float>(t, G->rot_cos, (jrot > 0 ? 1.f : -1.f) * G->rot_sin, G->bzc) != 0) return false;
  if (kf_prop<float>(t, ob.x[b], G->bzc) != 0) return false;
  // back to the physical tan(lambda) of the output convention
  t.p[3] *= sga;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (k != 3) t.C[ix(3, k)] *= sga;
  const int idx[4] = {0, 2, 3, 4};
  float dv[4], cs[10];
  const float* pb = ob.par + (size_t)b * 5;
  const float* cb = ob.cov + (size_t)b * 15;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    dv[i] = t.p[idx[i]] - pb[idx[i]];
#pragma unroll
    for (int j = 0; j <= i; ++j) cs[ix(i, j)] = t.C[ix(idx[i], idx[j])] + cb[ix(idx[i], idx[j])];
  }
  const bool ok = chi2_4(dv, cs, chi2) && chi2 <= kChi2Mem;
  const float zu = G->zunit;
  const float zb = (float)(ob.zref[b] - ob.zref[a]) * zu + pb[1];
  zmRel = 0.5f * (t.p[1] + zb);
  zmVar = 0.25f * (t.C[ix(1, 1)] + cb[ix(1, 1)]);
  const int zmx = max(ea.zmax, eb.zmax);
  return !cuts || (ok && zmRel >= (float)(zmx - ob.zref[a]) * zu - kMemZTol);
}

// Signed transverse arc length to the closest approach to the origin of the
// circle through (x0, y0) with direction sin(phi) = snp and curvature k:
// atan2(k t, 1 - k d) / k with t = -(x0 cos + y0 sin), d = x0 sin - y0 cos
// (t itself at k = 0).
__device__ inline float dca_arc(float x0, float y0, float snp, float k) {
  const float csp = sqrtf((1.f - snp) * (1.f + snp));
  const float t = -(x0 * csp + y0 * snp), d = x0 * snp - y0 * csp;
  if (k == 0.f) return t;
  return atan2f(k * t, 1.f - k * d) / k;
}

}  // namespace

__global__ void k_cont_keys(const int* __restrict__ nTrkDev, OutBufs ob, MergeBufs mb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nTrkDev) return;
  const Ends e = load_ends(ob, t);
  mb.next[t] = -1;
  mb.prev[t] = -1;
  mb.keyOut[t] = inner_piece(ob, t, e) ? 1 : -1;
  int ki = -1;
  if (outer_piece(ob, t, e)) {
    ki = (e.tf * kNSec + e.sin) * 2;
    atomicAdd(&mb.listCnt[ki], 1);
  }
  mb.keyIn[t] = ki;
}

__global__ void k_cont_fill(const int* __restrict__ nTrkDev, OutBufs ob, MergeBufs mb, int* __restrict__ cursor) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nTrkDev) return;
  const int k = mb.keyIn[t];
  if (k < 0) return;
  const int slot = mb.listStart[k] + atomicAdd(&cursor[k], 1);
  mb.listItems[slot] = t;
  mb.listKey[slot] = ob.ends[t].z;
}

// One thread per inner piece: the outer pieces of the three sector angles
// around its end on the other side, inside the first-zeta window.  Pairs go
// to mb.pairs with the TF's first key as their group.
__global__ void __launch_bounds__(128) k_cont_pairs(const int* __restrict__ nTrkDev, OutBufs ob, MergeBufs mb,
                                                    const GeomConst* __restrict__ G, unsigned* __restrict__ err) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= *nTrkDev || mb.keyOut[a] < 0) return;
  const Ends ea = load_ends(ob, a);
  const int other = ea.sout < 18 ? 18 : 0;
  for (int d = -1; d <= 1; ++d) {
    const int sb = other + (ea.sout % 18 + d + 18) % 18;
    const int key = (ea.tf * kNSec + sb) * 2;
    int lo = mb.listStart[key], hi = mb.listStart[key + 1];
    if (lo == hi) continue;
    {
      int l = lo, h = hi;
      while (l < h) {
        const int m = (l + h) >> 1;
        if (mb.listKey[m] < ea.zout - kMemDZetaUnits) l = m + 1;
        else h = m;
      }
      const int first = l;
      h = hi;
      while (l < h) {
        const int m = (l + h) >> 1;
        if (mb.listKey[m] <= ea.zout + kMemDZetaUnits) l = m + 1;
        else h = m;
      }
      lo = first;
      hi = l;
    }
    for (int q = lo; q < hi; ++q) {
      const int b = mb.listItems[q];
      const Ends eb = load_ends(ob, b);
      float c2, zm, zv;
      if (!membrane_match(ob, G, a, ea, b, eb, true, c2, zm, zv)) continue;
      const int slot = atomicAdd(mb.pairCount, 1);
      if (slot < mb.pairCap)
        mb.pairs[slot] = make_float4(c2, __int_as_float(a), __int_as_float(b), __int_as_float(ea.tf * kNSec * 2));
      else
        atomicOr(err, kErrMembrane);
    }
  }
}

__global__ void k_cont_t0(const int* __restrict__ nTrkDev, OutBufs ob, MergeBufs mb, const GeomConst* __restrict__ G,
                          const TFDesc* __restrict__ tfs, const double* __restrict__ coll,
                          const int* __restrict__ trkTfBegin) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *nTrkDev) return;
  const Ends e = load_ends(ob, t);
  const double zu = G->zunit_d, vd = G->vd_d;
  double lo = ((double)e.zmax * zu - 250.0) / vd;
  double hi = (double)e.zmin * zu / vd;
  double t0, er;
  int mate = -1;
  const int a = mb.prev[t] >= 0 ? mb.prev[t] : (mb.next[t] >= 0 ? t : -1);
  if (a >= 0) {
    // linked: the inner piece a and the outer piece b
    const int b = mb.next[a];
    mate = (a == t) ? b : a;
    const Ends ea = (a == t) ? e : load_ends(ob, a);
    const Ends eb = (a == t) ? load_ends(ob, b) : e;
    float c2, zm = 0.f, zv = 0.f;
    membrane_match(ob, G, a, ea, b, eb, false, c2, zm, zv);
    t0 = ((double)ob.zref[a] * zu + (double)zm - 250.0) / vd;
    er = sqrt((double)zv) / vd;
    const Ends& eo = (a == t) ? eb : ea;
    lo = fmax(lo, ((double)eo.zmax * zu - 250.0) / vd);
    hi = fmin(hi, (double)eo.zmin * zu / vd);
    ob.flags[t] |= 8;
  } else {
    const float* p = ob.par + (size_t)t * 5;
    const float* C = ob.cov + (size_t)t * 15;
    if (!(fabsf(p[2]) < 1.f)) {
      t0 = 0.5 * (lo + hi);
      er = 0.5 * (hi - lo);
    } else {
      const float side = (float)side_of(ob.sector[t]);
      const float s = dca_arc(ob.x[t], p[0], p[2], p[4] * G->bzc);
      const float dzds = -side * p[3];
      const float zrel = p[1] + dzds * s;
      t0 = ((double)ob.zref[t] * zu + (double)zrel - 250.0) / vd;
      t0 = fmin(fmax(t0, lo), hi);
      const float c13 = -side * C[ix(1, 3)];
      float var = C[ix(1, 1)] + 2.f * s * c13 + s * s * C[ix(3, 3)];
      if (!(var >= 0.f)) var = 0.f;
      er = sqrt((double)var + (double)kSigmaZv * kSigmaZv) / vd;
    }
  }
  // nearest compatible interaction time (sorted per TF; ties: the earlier)
  int best = -1;
  const TFDesc& d = tfs[e.tf];
  if (d.nColl > 0) {
    const double* T = coll + d.collBase;
    const int n = d.nColl;
    auto lower = [&](double v, int l, int h) {
      while (l < h) {
        const int m = (l + h) >> 1;
        if (T[m] < v) l = m + 1;
        else h = m;
      }
      return l;
    };
    const int ia = lower(lo - kT0Slack, 0, n);
    int ib = ia;
    {
      int h = n;
      const double v = hi + kT0Slack;
      while (ib < h) {
        const int m = (ib + h) >> 1;
        if (T[m] <= v) ib = m + 1;
        else h = m;
      }
    }
    if (ia < ib) {
      const int j = lower(t0, ia, ib);
      int k;
      if (j == ia) k = ia;
      else if (j == ib) k = ib - 1;
      else k = (t0 - T[j - 1] <= T[j] - t0) ? j - 1 : j;
      best = lower(T[k], ia, k + 1);  // the first of equal times
    }
  }
  ob.t0[t] = (float)t0;
  ob.t0err[t] = (float)er;
  ob.t0lo[t] = (float)lo;
  ob.t0hi[t] = (float)hi;
  ob.mate[t] = mate >= 0 ? mate - trkTfBegin[e.tf] : -1;
  ob.coll[t] = best;
}

void launch_continuous(int nTrk, const int* nTrkDev, int nKeys, OutBufs ob, MergeBufs mb, const GeomConst* G,
                       const TFDesc* tfs, const double* coll, const int* trkTfBegin, unsigned* err, int* scratch,
                       cudaStream_t st) {
  if (nTrk <= 0) return;
  const int g = (nTrk + 255) / 256;
  cudaMemsetAsync(mb.listCnt, 0, sizeof(int) * (nKeys + 1), st);
  cudaMemsetAsync(mb.pairCount, 0, sizeof(int), st);
  k_cont_keys<<<g, 256, 0, st>>>(nTrkDev, ob, mb);
  scan_exclusive(mb.listCnt, mb.listStart, nKeys, &mb.cnt->nKeys, scratch, st);
  cudaMemsetAsync(mb.listCnt, 0, sizeof(int) * (nKeys + 1), st);
  k_cont_fill<<<g, 256, 0, st>>>(nTrkDev, ob, mb, mb.listCnt);
  g_launch_count += 2;
  launch_list_sort(nKeys, mb, st);
  k_cont_pairs<<<(nTrk + 127) / 128, 128, 0, st>>>(nTrkDev, ob, mb, G, err);
  ++g_launch_count;
  launch_merge_select(mb.pairCap, nKeys, mb, scratch, st);
  k_cont_t0<<<g, 256, 0, st>>>(nTrkDev, ob, mb, G, tfs, coll, trkTfBegin);
  ++g_launch_count;
}

}  // namespace o2tpc
