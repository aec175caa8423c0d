// o2tpc_internal.cuh - shared device definitions of the tracker kernels.
//
// Geometry, tracking cuts and the Kalman-filter building blocks used by the
// kernels in k_*.cu.  All tracking decisions up to the start hits are
// integer; the track fit runs in FP32 (templated so that the final refit can
// redo a track in FP64 when its FP32 covariance stops being positive
// definite).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace o2tpc {

// ------------------------------------------------------------ geometry
constexpr int kNSec = 36;
constexpr int kNRow = 152;
constexpr int kRowsPerTF = kNSec * kNRow;  // 5472

// ------------------------------------------------------ integer seeding
constexpr int kCellY = 320;        // grid cell width along y: 2 cm in 1/160 cm
constexpr int kHitsPerCell = 4;    // target occupancy of a grid cell
constexpr int kMaxNz = 1 << 20;    // cells along zeta per row, at most
constexpr int kWinY = 240;         // neighbour window |dy| <= 1.5 cm
constexpr int kWinZ = 248;         // neighbour window |dzeta| <= 2.0 cm
constexpr int kWeightY = 2077;     // 6 sigma_zeta^2 in units^2: weight of the y term
constexpr int kWeightZ = 1536;     // 6 sigma_y^2 in units^2: weight of the zeta term
constexpr int kMaxMetric = 16 * 1536 * 2077;  // 2-dof chi2 <= 16, scaled

// ---------------------------------------------------------- track fit
constexpr float kSigY = 0.1f;
constexpr float kSigZ = 0.15f;
// Angle-dependent cluster errors (optional model): the variances grow by
// (L tan phi)^2 / 12 along y and (L tan lambda)^2 / 12 along the drift, L the
// pad length (the row pitch, 160/151 cm).
constexpr double kLpad2_12 = (160.0 / 151.0) * (160.0 / 151.0) / 12.0;
constexpr int kMaxMiss = 4;        // consecutive rows without a hit before stopping
constexpr int kMinHits = 10;       // tracklet / sector-track minimum
constexpr float kChi2Follow = 18.f;
constexpr float kSinFollow = 0.95f;
constexpr float kSinProp = 0.999f;
constexpr float kEdgeBand = 5.f;   // border-track band for merging, cm
constexpr float kMergeDZeta = 20.f;
constexpr float kChi2Merge = 30.f;

// Per-run constants in constant memory (set by the host once per context).
struct GeomConst {
  float rowx[kNRow];
  double rowx_d[kNRow];
  float pitch;      // pad-row spacing 160/151 cm: transport steps between rows
  double pitch_d;
  int angErr;       // 1: angle-dependent cluster errors
  int rowStep2;     // 1: the NeighboursFinder also links across one missing row
  int npads[kNRow];
  float sec_alpha[18];
  float tan10;
  float rot_cos, rot_sin;      // cos / sin of the 20 degree sector pitch
  double rot_cos_d, rot_sin_d;
  float bzc;        // -0.00299792458 * Bz (1/cm per GeV^-1)
  float zunit;      // cm per drift-time unit (0.003125 us * v_drift)
  float kz;         // 1 / zunit as float (float-input quantisation)
  double bzc_d, zunit_d;
  double vd_d;      // drift velocity, cm/us
};

// ------------------------------------------------------------ tables
// Per-row grid, 32 bytes.
struct RowGrid {
  int start;     // first sorted hit of the row (batch-global)
  int count;
  int cellBase;  // first cell of the row in cellStart[]
  int ny, nz, cz, zmin;
  int pad;
};

// Per-TF descriptor of a batch.
struct TFDesc {
  const void* in0;   // FLOAT: sector (uint8) / FIXED: packed records
  const void* in1;   // FLOAT: row (uint8)
  const float* y;    // FLOAT
  const float* z;    // FLOAT: apparent z, or null
  const float* time; // FLOAT without z: drift time (us)
  int format;
  int n;             // clusters
  int inBase;        // first batch-global input index of this TF
  int tileBase;      // first tile of this TF
  int nTiles;
  int nColl;         // interaction times of this TF (ascending, us)
  int collBase;      // first of them in the batch's array
};

// Fills the geometry table for a field of bz tesla and a drift velocity of vd
// cm/us (host side; defined in o2tpc_capi.cu, used by every entry point).
void fill_geom(GeomConst& g, double bz, double vd);

// Device error word bits
enum : unsigned { kErrInput = 1u, kErrOverflow = 2u, kErrTimeout = 4u, kErrMembrane = 8u };

// ------------------------------------------------------------ helpers
// floor(a / b) for b > 0 in 32-bit arithmetic.
__host__ __device__ inline int floordiv_i32(int a, int b) {
  const int q = a / b;
  return (q * b > a) ? q - 1 : q;
}

__device__ inline int cell_iy(const RowGrid& g, int npads, int yu) {
  int half = 32 * npads;
  int iy = floordiv_i32(yu + half, kCellY);
  return iy < 0 ? 0 : (iy > g.ny - 1 ? g.ny - 1 : iy);
}

// Cell row of a drift coordinate: floor((v - zmin) / cz), -1 below the row's
// range.  v - zmin can exceed the int32 range (|v|, |zmin| < 2^31), so the
// difference and the division are unsigned.
// The quotient is estimated in single precision and corrected by one step:
// the estimate is within one of the true quotient for quotients up to 2^20
// (nz never exceeds that); larger ones are clamped to nz, which callers clamp
// further.
__device__ inline int cell_iz_floor(int v, const RowGrid& g) {
  if (v < g.zmin) return -1;
  const unsigned x = (unsigned)v - (unsigned)g.zmin, cz = (unsigned)g.cz, nz = (unsigned)g.nz;
  const float qe = __fdividef((float)x, (float)cz);
  unsigned q = qe >= (float)nz ? nz : (unsigned)qe;
  if ((unsigned long long)q * cz > x) --q;
  else if (q < nz && (unsigned long long)(q + 1) * cz <= x) ++q;
  return (int)q;
}

// Cell rectangle of row g overlapping [ylo,yhi] x [zlo,zhi]; false if empty.
// Coordinates are integer units inside the int32 range (y windows within a
// few 10^6, z windows within +-2.1e9), so 32-bit arithmetic suffices.
__device__ inline bool cell_range(const RowGrid& g, int npads, int ylo, int yhi, int zlo, int zhi, int& iy0,
                                  int& iy1, int& iz0, int& iz1) {
  if (g.count == 0) return false;
  const int half = 32 * npads;
  const int qa = floordiv_i32(ylo + half, kCellY);
  const int qb = floordiv_i32(yhi + half, kCellY);
  iy0 = qa < 0 ? 0 : (qa > g.ny - 1 ? g.ny - 1 : qa);
  iy1 = qb < 0 ? 0 : (qb > g.ny - 1 ? g.ny - 1 : qb);
  int qza = cell_iz_floor(zlo, g);
  int qzb = cell_iz_floor(zhi, g);
  if (qza < 0) qza = 0;
  if (qzb > g.nz - 1) qzb = g.nz - 1;
  if (qza > qzb) return false;
  iz0 = qza;
  iz1 = qzb;
  return true;
}

__device__ inline int upper_bound_i32(const int* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (a[m] <= v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// ------------------------------------------------- Kalman building blocks
// State (y, zeta, sin phi, t = dzeta/ds_T, q/pT) at local x; covariance as
// lower triangle (yy, zy, zz, sy, sz, ss, ty, tz, ts, tt, qy, qz, qs, qt, qq).
template <typename T>
struct KState {
  T x;
  T p[5];
  T C[15];
};

__host__ __device__ constexpr int ix(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

template <typename T>
__device__ inline T kf_sqrt(T v);
template <>
__device__ inline float kf_sqrt<float>(float v) { return sqrtf(v); }
template <>
__device__ inline double kf_sqrt<double>(double v) { return sqrt(v); }
template <typename T>
__device__ inline T kf_asin(T v);
template <>
__device__ inline float kf_asin<float>(float v) { return asinf(v); }
template <>
__device__ inline double kf_asin<double>(double v) { return asin(v); }

// Cluster variances (y, zeta) for a track with the state's angles: kSigY^2,
// kSigZ^2, plus with the angle-dependent model (angErr) the pad-length terms
// kLpad2_12 * tan^2(phi), tan^2(phi) = s^2 / (1 - s^2) from s = sin(phi), and
// kLpad2_12 * t^2 (t = dzeta/ds, |t| = tan(lambda)).
template <typename T>
__device__ inline void meas_var(int angErr, const KState<T>& s, T& vy, T& vz) {
  vy = T(kSigY) * T(kSigY);
  vz = T(kSigZ) * T(kSigZ);
  if (angErr) {
    const T s2 = s.p[2] * s.p[2];
    const T tan2 = s2 < T(1) ? s2 / (T(1) - s2) : T(1e6);
    vy += T(kLpad2_12) * tan2;
    vz += T(kLpad2_12) * s.p[3] * s.p[3];
  }
}

template <typename T>
__device__ inline void kf_reset(KState<T>& s, T x, T y, T z, T sphi, T t, T q) {
  s.x = x;
  s.p[0] = y; s.p[1] = z; s.p[2] = sphi; s.p[3] = t; s.p[4] = q;
#pragma unroll
  for (int i = 0; i < 15; ++i) s.C[i] = T(0);
  s.C[0] = T(kSigY) * T(kSigY);
  s.C[2] = T(kSigZ) * T(kSigZ);
  s.C[5] = T(0.04);
  s.C[9] = T(0.25);
  s.C[14] = T(400);
}

// C <- J C J^T for J = identity plus the listed off-diagonal terms.
template <typename T>
__device__ inline void kf_sandwich(T* C, const T J[5][5]) {
  T M[5][5], A[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) M[i][j] = C[ix(i, j)];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) s += J[i][k] * M[k][j];
      A[i][j] = s;
    }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T s = T(0), s2 = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) { s += A[i][k] * J[j][k]; s2 += A[j][k] * J[i][k]; }
      C[ix(i, j)] = T(0.5) * (s + s2);
    }
}

// C <- J C J^T for the transport Jacobian J = I + a02 e0e2' + a04 e0e4' +
// a12 e1e2' + a13 e1e3' + a14 e1e4' + a24 e2e4' (the only non-zero
// off-diagonal terms), written out: T = J C for rows 0-2 (rows 3, 4 of T are
// those of C), then C' = T J^T on the lower triangle.
template <typename T>
__device__ inline void kf_sandwich_transport(T* C, T a02, T a04, T a12, T a13, T a14, T a24) {
  T c[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) c[i][j] = C[ix(i, j)];
  T t0[5], t1[5], t2[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    t0[k] = c[0][k] + a02 * c[2][k] + a04 * c[4][k];
    t1[k] = c[1][k] + a12 * c[2][k] + a13 * c[3][k] + a14 * c[4][k];
    t2[k] = c[2][k] + a24 * c[4][k];
  }
  C[ix(0, 0)] = t0[0] + a02 * t0[2] + a04 * t0[4];
  C[ix(1, 0)] = t1[0] + a02 * t1[2] + a04 * t1[4];
  C[ix(1, 1)] = t1[1] + a12 * t1[2] + a13 * t1[3] + a14 * t1[4];
  C[ix(2, 0)] = t2[0] + a02 * t2[2] + a04 * t2[4];
  C[ix(2, 1)] = t2[1] + a12 * t2[2] + a13 * t2[3] + a14 * t2[4];
  C[ix(2, 2)] = t2[2] + a24 * t2[4];
  C[ix(3, 0)] = c[3][0] + a02 * c[3][2] + a04 * c[3][4];
  C[ix(3, 1)] = c[3][1] + a12 * c[3][2] + a13 * c[3][3] + a14 * c[3][4];
  C[ix(3, 2)] = c[3][2] + a24 * c[3][4];
  C[ix(4, 0)] = c[4][0] + a02 * c[4][2] + a04 * c[4][4];
  C[ix(4, 1)] = c[4][1] + a12 * c[4][2] + a13 * c[4][3] + a14 * c[4][4];
  C[ix(4, 2)] = c[4][2] + a24 * c[4][4];
}

// Helix transport to x2 in a uniform field: d(sin phi)/dx = k = (q/pT) bzc;
// dy = dx (s1+s2)/(c1+c2); transverse path ds = 2 asin(|k| chord/2)/|k|
// (the chord when |k| chord < 1e-6), signed like dx; dzeta = t ds.
// Jacobian: exact y and sin(phi) rows; d(ds)/d(sin phi) exact; d(ds)/dk as
// a three-point Simpson integral of its cancellation-free integrand when
// |k dx| < 0.05, else (dx/c2 - ds)/k.  Returns 0, or -1 if |sin phi| would
// reach kSinProp.
// One transport step's increments and Jacobian terms from parameters p
// (y, zeta, sin phi, t, q/pT) over dx; -1 if |sin phi| would reach kSinProp.
template <typename T>
struct PropStep {
  T dy, dzeta, s2, a02, a04, a12, a13, a14, a24;
};
template <typename T>
__device__ inline int kf_prop_step(const T* p, T dx, T bzc, PropStep<T>& o) {
  T s1 = p[2], q = p[4], tz = p[3];
  T k = q * bzc;
  T s2 = s1 + k * dx;
  if (fabs(s1) >= T(kSinProp) || fabs(s2) >= T(kSinProp)) return -1;
  T c1 = kf_sqrt<T>((T(1) - s1) * (T(1) + s1));
  T c2 = kf_sqrt<T>((T(1) - s2) * (T(1) + s2));
  T cc = c1 + c2;
  // reciprocals once, products after (the divisions dominate the cost)
  const T icc = T(1) / cc, ic1 = T(1) / c1, ic2 = T(1) / c2;
  T dy = dx * (s1 + s2) * icc;
  T chord = kf_sqrt<T>(dx * dx + dy * dy);
  T ak = fabs(k) * chord;
  // arc length 2 asin(ak/2)/|k|.  In single precision, for ak/2 = h < 0.05
  // the Taylor series asin(h)/h = 1 + h^2/6 + 3h^4/40 + ... truncated after
  // the h^4 term is exact to 7e-10 relative (next term 5h^6/112), below the
  // precision of the result.  Double precision keeps asin.
  const T h = T(0.5) * ak;
  T ds;
  if (sizeof(T) == 4 && h < T(0.05)) {
    const T h2 = h * h;
    ds = chord * (T(1) + h2 * (T(1.0 / 6.0) + h2 * T(3.0 / 40.0)));
  } else if (ak < T(1e-6)) {
    ds = chord;
  } else {
    ds = T(2) * kf_asin<T>(h) / fabs(k);
  }
  if (dx < T(0)) ds = -ds;
  T sm = s1 + T(0.5) * k * dx;
  T cm = kf_sqrt<T>((T(1) - sm) * (T(1) + sm));
  T f1 = dx * (s1 + s2) * ic1 * ic2 * icc;
  T fm = T(0.5) * dx * (sm + s2) * ic2 / (cm * (cm + c2));
  T ddsdk = (fabs(k * dx) < T(0.05)) ? dx * (f1 + T(4) * fm) * T(1.0 / 6.0) : (dx * ic2 - ds) / k;
  const T a02 = dx * (T(2) * cc + (s1 + s2) * (s1 * ic1 + s2 * ic2)) * icc * icc;
  const T a04 = dx * dx * bzc * (cc + (s1 + s2) * s2 * ic2) * icc * icc;
  const T a12 = tz * f1;
  const T a13 = ds;
  const T a14 = tz * bzc * ddsdk;
  const T a24 = dx * bzc;
  o.dy = dy;
  o.dzeta = tz * ds;
  o.s2 = s2;
  o.a02 = a02;
  o.a04 = a04;
  o.a12 = a12;
  o.a13 = a13;
  o.a14 = a14;
  o.a24 = a24;
  return 0;
}

template <typename T>
__device__ inline int kf_prop_dx(KState<T>& s, T x2, T dx, T bzc) {
  if (dx == T(0)) return 0;
  PropStep<T> o;
  if (kf_prop_step<T>(s.p, dx, bzc, o) != 0) return -1;
  s.p[0] += o.dy;
  s.p[1] += o.dzeta;
  s.p[2] = o.s2;
  s.x = x2;
  kf_sandwich_transport<T>(s.C, o.a02, o.a04, o.a12, o.a13, o.a14, o.a24);
  return 0;
}

// The FP64 fallback's transport: the step's geometry (increments and
// Jacobian terms) in single precision, as on the FP32 path, applied to the
// double-precision state, and the covariance propagated in double.  Double
// precision is needed only where the FP32 covariance lost positive
// definiteness; the transcendental geometry stays single precision, where a
// GPU runs it fast.
__device__ inline int kf_prop_dx_cov64(KState<double>& s, double x2, float dx, float bzc) {
  if (dx == 0.f) return 0;
  float pf[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) pf[i] = (float)s.p[i];
  PropStep<float> o;
  if (kf_prop_step<float>(pf, dx, bzc, o) != 0) return -1;
  s.p[0] += (double)o.dy;
  s.p[1] += (double)o.dzeta;
  s.p[2] += s.p[4] * (double)bzc * (double)dx;
  s.x = x2;
  kf_sandwich_transport<double>(s.C, o.a02, o.a04, o.a12, o.a13, o.a14, o.a24);
  return 0;
}

// Transport to x2 from a state at any x (after a frame rotation, or to another
// track's x): the step is the difference of the two positions.
template <typename T>
__device__ inline int kf_prop(KState<T>& s, T x2, T bzc) {
  return kf_prop_dx<T>(s, x2, x2 - s.x, bzc);
}

// Transport between pad rows r1 -> r2 of a state sitting on row r1.  The step
// (r2 - r1) * pitch carries one rounding; the difference of the two rounded
// row positions would carry up to 1.5e-5 cm in single precision, an error
// that dominates the FP32 curvature of short tracks (a 10-row stub's
// sagitta is a few 1e-3 cm).
template <typename T>
__device__ inline int kf_prop_row(KState<T>& s, int r1, int r2, const GeomConst* __restrict__ G, T bzc) {
  const T pitch = sizeof(T) == 8 ? (T)G->pitch_d : (T)G->pitch;
  const T x2 = sizeof(T) == 8 ? (T)G->rowx_d[r2] : (T)G->rowx[r2];
  return kf_prop_dx<T>(s, x2, (T)(r2 - r1) * pitch, bzc);
}

// Pad row of a state whose x is a row position (within its rounding).
__device__ inline int row_of_x(float x) { return __float2int_rn((x - 85.f) * (151.f / 160.f)); }

// Moves a fit's y origin yref (integer units of 1/160 cm) in whole
// centimetres to within half a centimetre of the hit at yu, and the state's y
// (cm, relative to the origin) with it.  A shift by whole centimetres is an
// exact number, so the state only takes the rounding of a value below ~1 cm;
// the fits then never hold y values of several cm, whose rounding (2e-7 cm at
// 4 cm) would show in the curvature of short tracks.
// Moves a fit's drift origin zref (integer units) to the hit at zu, and the
// state's zeta (cm, relative to the origin) with it: the fit then only holds
// zeta values of about a row step, and the rounding of the tens of cm a long
// steep track spans does not build up along it.  The shift itself carries one
// rounding of a value of that row step's size.
template <typename T>
__device__ inline void recentre_z(T& z, int& zref, int zu, T zunit) {
  const int d = zu - zref;
  if (d != 0) {
    z -= (T)d * zunit;
    zref = zu;
  }
}

template <typename T>
__device__ inline void recentre_y(T& y, int& yref, int yu) {
  const int m = floordiv_i32(yu - yref + 80, 160);
  if (m != 0) {
    y -= (T)m;
    yref += 160 * m;
  }
}

// Kalman update with a (y, zeta) measurement of variances (vy, vz).
template <typename T>
__device__ inline int kf_update_v(KState<T>& s, T ym, T zm, T vy, T vz, T* chi2) {
  T* C = s.C;
  T r0 = ym - s.p[0], r1 = zm - s.p[1];
  T S00 = C[0] + vy, S01 = C[1], S11 = C[2] + vz;
  T det = S00 * S11 - S01 * S01;
  if (!(det > T(0))) return -1;
  const T idet = T(1) / det;
  T I00 = S11 * idet, I01 = -S01 * idet, I11 = S00 * idet;
  if (chi2) *chi2 = r0 * r0 * I00 + T(2) * r0 * r1 * I01 + r1 * r1 * I11;
  T Cy[5], Cz[5], K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) { Cy[i] = C[ix(i, 0)]; Cz[i] = C[ix(i, 1)]; }
#pragma unroll
  for (int i = 0; i < 5; ++i) { K0[i] = Cy[i] * I00 + Cz[i] * I01; K1[i] = Cy[i] * I01 + Cz[i] * I11; }
#pragma unroll
  for (int i = 0; i < 5; ++i) s.p[i] += K0[i] * r0 + K1[i] * r1;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ix(i, j)] -= K0[i] * Cy[j] + K1[i] * Cz[j];
  return 0;
}

// Kalman update with the cluster variances of the error model at the
// predicted state's angles.
template <typename T>
__device__ inline int kf_update(KState<T>& s, T ym, T zm, T* chi2, int angErr) {
  T vy, vz;
  meas_var<T>(angErr, s, vy, vz);
  return kf_update_v<T>(s, ym, zm, vy, vz, chi2);
}

// The (y, zeta) entries of a fresh covariance: the cluster variances at the
// state's angles.
template <typename T>
__device__ inline void kf_meas_cov(KState<T>& s, int angErr) {
  meas_var<T>(angErr, s, s.C[0], s.C[2]);
}

// Frame rotation by dalpha (cos ca, sin sa): new alpha = old alpha + dalpha.
// Parameters follow the rigid rotation; covariance Jacobian: dy'/dy = c/c',
// dzeta'/dy = -t sa / c', d(sin phi')/dy = -k sa, d(sin phi')/d(sin phi) = c'/c.
template <typename T>
__device__ inline int kf_rotate(KState<T>& s, T ca, T sa, T bzc) {
  T sp = s.p[2];
  if (fabs(sp) >= T(kSinProp)) return -1;
  T c = kf_sqrt<T>((T(1) - sp) * (T(1) + sp));
  T s2 = sp * ca - c * sa, c2 = c * ca + sp * sa;
  if (c2 <= T(0) || fabs(s2) >= T(kSinProp)) return -1;
  T x = s.x, y = s.p[0];
  T J[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) J[i][j] = (i == j) ? T(1) : T(0);
  J[0][0] = c / c2;
  J[1][0] = -s.p[3] * sa / c2;
  J[2][0] = -s.p[4] * bzc * sa;
  J[2][2] = c2 / c;
  s.x = x * ca + y * sa;
  s.p[0] = -x * sa + y * ca;
  s.p[2] = s2;
  kf_sandwich<T>(s.C, J);
  return 0;
}

// FP32 positive-definiteness test of the final refit: every C_ii > 0 and
// every C_ij^2 < C_ii C_jj.
template <typename T>
__device__ inline bool kf_cov_ok(const T* C) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (!(C[ix(i, i)] > T(0))) return false;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      T v = C[ix(i, j)];
      if (!(v * v < C[ix(i, i)] * C[ix(j, j)])) return false;
    }
  return true;
}

}  // namespace o2tpc
