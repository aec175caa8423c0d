/*
 * o2tpc_oracle.c - FP64, single-threaded CPU oracle of the TPC Time-Frame
 * tracker.
 *
 * TEST INFRASTRUCTURE ONLY: this file is the reference the CUDA path is
 * checked against.  Only the tests, the package entry's smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes.  The paper places TPC track reconstruction over a whole
 * continuous-readout Time Frame at the centre of the synchronous processing
 * (Sec. 2.1: the dominant workload; Sec. 2.3: derived from the Run-2 HLT
 * tracker, handling continuous readout without a priori z and a five-fold
 * occupancy; Sec. 2: the Time Frame is the processing unit).  It does not
 * spell out the algorithm, so every step below follows one written-down
 * reading of a cellular-automaton seeding plus Kalman-filter following
 * tracker, step by step, in plain code:
 *
 *   1. ingest: clusters -> integer y_u (1/160 cm) and zeta_u (1/64 time bin)
 *   2. per (sector,row) grid and stable sort by (sector,row,cell,input index)
 *   3. NeighboursFinder: best (up,down) pair by an integer straightness metric
 *   4. NeighboursCleaner: keep reciprocal links only (snapshot semantics)
 *   5. StartHitsFinder: heads of chains of >= 3 hits
 *   6. TrackletConstructor: Kalman fit of the chain, following up then down
 *   7. TrackletSelector: hit ownership by the longest tracklet, gap split
 *   8. sector-to-sector merger of border tracks (chi2 on 5 parameters)
 *   9. final inward refit, output at the innermost cluster
 *
 * Floating point is double everywhere except the FP32 quantisation of float
 * input, which is part of the input format's definition.  Pins: see
 * tests/test_oracle_*.py (brute-force neighbour search, sort invariants, helix
 * closed form, least-squares fit, pulls, efficiency, merge truth).
 */
#include "o2tpc_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ constants */
#define O_NSEC 36
#define O_NROW 152
#define O_NROWS (O_NSEC * O_NROW)
#define O_PI 3.14159265358979323846
#define O_CY 320            /* grid cell width in y, units (2 cm)               */
#define O_T 4               /* target hits per cell                              */
#define O_NZMAX (1 << 20)   /* max cells along zeta per row                      */
#define O_WY 240            /* neighbour window |dy| (1.5 cm), units             */
#define O_WZ 248            /* neighbour window |dzeta| (2.0 cm), units          */
#define O_AY 2077LL         /* weight of the y term  (6 sigma_z^2 in units^2)    */
#define O_AZ 1536LL         /* weight of the zeta term (6 sigma_y^2 in units^2)  */
#define O_DMAX (16LL * 1536LL * 2077LL) /* chi2 <= 16 for 2 dof                   */
#define O_SY 0.1            /* cluster error y, cm                               */
#define O_SZ 0.15           /* cluster error zeta, cm                            */
#define O_G 4               /* max consecutive missed rows                       */
#define O_NMIN 10           /* min hits of a tracklet / sector track             */
#define O_CHI2_FOLLOW 18.0
#define O_SIN_FOLLOW 0.95
#define O_SIN_PROP 0.999
#define O_EDGE 5.0          /* border-track band, cm                             */
#define O_DZETA_PRE 20.0    /* merge prefilter on endpoint zeta, cm              */
#define O_CHI2_MERGE 30.0
/* Angle-dependent cluster errors (reading, optional): a track crossing the
 * pad row at an angle spreads its charge over the pad length L (the row
 * pitch, 160/151 cm) times tan(phi) along y and times tan(lambda) along the
 * drift; the centroid's variance grows by (L tan)^2 / 12 (a uniform spread
 * of that width). */
#define O_LPAD2_12 ((160.0 / 151.0) * (160.0 / 151.0) / 12.0)

static double o_rowx(int r) { return 85.0 + (double)r * 160.0 / 151.0; }
static int o_npads(int r) { return (int)floor(2.0 * o_rowx(r) * tan(10.0 * O_PI / 180.0) / 0.4); }
static double o_alpha(int s) { return ((double)(s % 18) * 20.0 + 10.0) * O_PI / 180.0; }
static int o_side(int s) { return s < 18 ? 1 : -1; }
static double o_tan10(void) { return tan(10.0 * O_PI / 180.0); }
static int64_t o_floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }

/* Initial covariance of every fit: the first hit's (y, zeta) errors, and
 * loose priors on the seeded sin(phi) (0.2), t (0.5) and q/pT (20, i.e. pT
 * down to 0.05 GeV).  A sin(phi) prior much wider than 0.2 makes the first
 * updates nearly singular, which single precision cannot follow. */
static const double O_CINIT[15] = {O_SY * O_SY, 0, O_SZ * O_SZ, 0, 0, 0.04, 0, 0, 0, 0.25, 0, 0, 0, 0, 400.0};
static int o_ix(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

/* ------------------------------------------------------------- result */
typedef struct { double x, p[5], C[15]; } ost;

typedef struct { const char* name; const void* ptr; int64_t n; int32_t type; } o_field;

struct oracle_result {
  int64_t n, nsel;
  double zunit, bzc;
  int angerr;   /* angle-dependent cluster errors */
  int rowstep2; /* NeighboursFinder also links across one missing pad row */
  /* per input cluster */
  int32_t *yu, *zu, *rid;
  /* per sorted hit */
  int32_t *s_orig, *s_rid, *s_y, *s_z, *s_cell;
  /* per row */
  int32_t r_cnt[O_NROWS], r_zmin[O_NROWS], r_zmax[O_NROWS], r_ny[O_NROWS], r_nz[O_NROWS];
  int64_t r_cz[O_NROWS];
  int64_t r_start[O_NROWS + 1], r_cellbase[O_NROWS + 1];
  int64_t* cell_start; /* [ncells + 1] */
  int64_t ncells;
  /* links */
  int32_t *up_raw, *dn_raw, *up, *dn;
  int32_t* starts; int64_t nstart;
  /* tracklets [nstart] */
  int32_t *tl_nhits, *tl_kept, *tl_zref; int64_t* tl_off; int32_t* tl_hits; int64_t tl_nh;
  double* tl_state; /* [nstart][21]: x, p5, C15 */
  /* sector tracks */
  int64_t nst;
  int32_t *st_sector, *st_tracklet, *st_zref; int64_t* st_off; int32_t* st_hits; int64_t st_nh;
  double *st_in, *st_out; /* [nst][21] */
  int32_t *st_next, *st_prev;
  /* merge candidates (for tests): [npair][3] a, b as int32 and chi2 */
  int64_t npair; int32_t* pair_ab; double* pair_chi2;
  /* final tracks */
  int64_t ntrk;
  int64_t* trk_off; int32_t* trk_cl; int64_t trk_ncl;
  double *trk_x, *trk_alpha, *trk_par, *trk_cov, *trk_chi2;
  int32_t *trk_ndf, *trk_sector, *trk_flags, *trk_zref, *trk_head, *trk_nseg;
  /* continuous readout: t0 (us), its error and bounds, membrane partner, collision */
  double *trk_t0, *trk_t0err, *trk_t0lo, *trk_t0hi;
  int32_t *trk_mate, *trk_coll;
  int64_t nmpair; int32_t* mpair_ab; double* mpair_chi2;
  /* compressed TF */
  uint8_t* ctf; int64_t ctf_bytes;
  o_field fields[80]; int nf;
};

/* ---------------------------------------------------- Kalman building blocks */
static void o_full(const double* c15, double M[5][5]) {
  for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) M[i][j] = c15[o_ix(i, j)];
}
static void o_pack(double M[5][5], double* c15) {
  for (int i = 0; i < 5; ++i) for (int j = 0; j <= i; ++j) c15[o_ix(i, j)] = 0.5 * (M[i][j] + M[j][i]);
}
static void o_sandwich(double J[5][5], double* c15) { /* C <- J C J^T */
  double C[5][5], T[5][5], R[5][5];
  o_full(c15, C);
  for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) { double s = 0; for (int k = 0; k < 5; ++k) s += J[i][k] * C[k][j]; T[i][j] = s; }
  for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) { double s = 0; for (int k = 0; k < 5; ++k) s += T[i][k] * J[j][k]; R[i][j] = s; }
  o_pack(R, c15);
}

/* Helix transport in a uniform field along z, in the sector frame: state
 * (y, zeta, sin phi, t = dzeta/ds_T, q/pT) at x; curvature k = (q/pT) * bzc
 * with bzc = -0.00299792458 * Bz (1/cm per GeV^-1), so that d(sin phi)/dx = k.
 *   sin phi_2 = sin phi_1 + k dx
 *   dy = dx (s1 + s2) / (c1 + c2)                       (exact on the circle)
 *   ds_T = 2 asin(|k| chord / 2) / |k|   (chord itself for |k| chord < 1e-6)
 *   dzeta = t ds_T
 * Jacobian: exact for y and sin phi; zeta row from
 *   d(ds_T)/d(sin phi_1) = dx (s1+s2) / (c1 c2 (c1+c2))                (exact)
 *   d(ds_T)/dk = integral_x1^x2 f(x) dx,
 *     f(x) = (x2 - x)(s2 + s(x)) / (c(x) c2 (c(x) + c2)),  s(x) = s1 + k (x - x1)
 * (the cancellation-free form of (dx/c2 - ds_T)/k), integrated with
 * Simpson's rule on x1, midpoint, x2 (f(x2) = 0) when |k dx| < 0.05 (relative
 * error < 1e-4 there), and (dx/c2 - ds_T)/k itself above.  No material, no
 * process noise. */
static int o_prop(ost* t, double x2, double bzc) {
  double dx = x2 - t->x;
  if (dx == 0.0) return 0;
  double s1 = t->p[2], q = t->p[4], tz = t->p[3];
  double k = q * bzc;
  double s2 = s1 + k * dx;
  if (fabs(s1) >= O_SIN_PROP || fabs(s2) >= O_SIN_PROP) return -1;
  double c1 = sqrt((1.0 - s1) * (1.0 + s1)), c2 = sqrt((1.0 - s2) * (1.0 + s2));
  double cc = c1 + c2;
  double dy = dx * (s1 + s2) / cc;
  double chord = sqrt(dx * dx + dy * dy);
  double ak = fabs(k) * chord;
  double ds = (ak < 1e-6) ? chord : 2.0 * asin(0.5 * ak) / fabs(k);
  if (dx < 0) ds = -ds;
  double J[5][5];
  memset(J, 0, sizeof(J));
  for (int i = 0; i < 5; ++i) J[i][i] = 1.0;
  J[0][2] = dx * (2.0 * cc + (s1 + s2) * (s1 / c1 + s2 / c2)) / (cc * cc);
  J[0][4] = dx * dx * bzc * (cc + (s1 + s2) * s2 / c2) / (cc * cc);
  J[1][2] = tz * dx * (s1 + s2) / (c1 * c2 * cc);
  J[1][3] = ds;
  double sm = s1 + 0.5 * k * dx, cm = sqrt((1.0 - sm) * (1.0 + sm));
  double f1 = dx * (s1 + s2) / (c1 * c2 * cc);
  double fm = 0.5 * dx * (sm + s2) / (cm * c2 * (cm + c2));
  double ddsdk = (fabs(k * dx) < 0.05) ? dx * (f1 + 4.0 * fm) / 6.0 : (dx / c2 - ds) / k;
  J[1][4] = tz * bzc * ddsdk;
  J[2][4] = dx * bzc;
  t->p[0] += dy;
  t->p[1] += tz * ds;
  t->p[2] = s2;
  t->x = x2;
  o_sandwich(J, t->C);
  return 0;
}

/* Measurement variances (y, zeta) of a cluster on a track with the state's
 * angles: the constant O_SY^2, O_SZ^2, plus with angerr the pad-length terms
 * (L tan(phi))^2 / 12 and (L tan(lambda))^2 / 12, tan^2(phi) = s^2 / (1 - s^2)
 * from sin(phi) = s, tan(lambda) = |dzeta/ds| = |t|. */
static void o_meas_var(int angerr, const ost* t, double* vy, double* vz) {
  *vy = O_SY * O_SY;
  *vz = O_SZ * O_SZ;
  if (angerr) {
    double s2 = t->p[2] * t->p[2];
    double tan2 = s2 < 1.0 ? s2 / (1.0 - s2) : 1e6;
    *vy += O_LPAD2_12 * tan2;
    *vz += O_LPAD2_12 * t->p[3] * t->p[3];
  }
}

/* Kalman update with a (y, zeta) measurement of variances (vy, vz). */
static int o_update_v(ost* t, double ym, double zm, double vy, double vz, double* chi2) {
  double* C = t->C;
  double r0 = ym - t->p[0], r1 = zm - t->p[1];
  double S00 = C[0] + vy, S01 = C[1], S11 = C[2] + vz;
  double det = S00 * S11 - S01 * S01;
  if (!(det > 0.0)) return -1;
  double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  if (chi2) *chi2 = r0 * r0 * I00 + 2.0 * r0 * r1 * I01 + r1 * r1 * I11;
  double Cy[5], Cz[5], K0[5], K1[5];
  for (int i = 0; i < 5; ++i) { Cy[i] = C[o_ix(i, 0)]; Cz[i] = C[o_ix(i, 1)]; }
  for (int i = 0; i < 5; ++i) { K0[i] = Cy[i] * I00 + Cz[i] * I01; K1[i] = Cy[i] * I01 + Cz[i] * I11; }
  for (int i = 0; i < 5; ++i) t->p[i] += K0[i] * r0 + K1[i] * r1;
  for (int i = 0; i < 5; ++i) for (int j = 0; j <= i; ++j) C[o_ix(i, j)] -= K0[i] * Cy[j] + K1[i] * Cz[j];
  return 0;
}

/* Kalman update with the constant cluster errors (O_SY, O_SZ). */
static int o_update(ost* t, double ym, double zm, double* chi2) {
  return o_update_v(t, ym, zm, O_SY * O_SY, O_SZ * O_SZ, chi2);
}

/* Rotation of the frame by dalpha (new alpha = old alpha + dalpha). */
static int o_rot(ost* t, double da, double bzc) {
  double ca = cos(da), sa = sin(da);
  double s = t->p[2];
  if (fabs(s) >= O_SIN_PROP) return -1;
  double c = sqrt((1.0 - s) * (1.0 + s));
  double s2 = s * ca - c * sa, c2 = c * ca + s * sa;
  if (c2 <= 0.0 || fabs(s2) >= O_SIN_PROP) return -1;
  double x = t->x, y = t->p[0];
  double J[5][5];
  memset(J, 0, sizeof(J));
  for (int i = 0; i < 5; ++i) J[i][i] = 1.0;
  J[0][0] = c / c2;
  J[1][0] = -t->p[3] * sa / c2;
  J[2][0] = -t->p[4] * bzc * sa;
  J[2][2] = c2 / c;
  t->x = x * ca + y * sa;
  t->p[0] = -x * sa + y * ca;
  t->p[2] = s2;
  o_sandwich(J, t->C);
  return 0;
}

static void o_init_state(ost* t, double x, double y, double z, double s, double tz, double q) {
  t->x = x; t->p[0] = y; t->p[1] = z; t->p[2] = s; t->p[3] = tz; t->p[4] = q;
  memcpy(t->C, O_CINIT, sizeof(O_CINIT));
}

/* ------------------------------------------------------- exported blocks */
static double o_bzc(double bz) { return -0.00299792458 * bz; }

int32_t oracle_propagate(double* x, double* p5, double* c15, double x2, double bz) {
  ost t; t.x = *x; memcpy(t.p, p5, 5 * sizeof(double)); memcpy(t.C, c15, 15 * sizeof(double));
  int rc = o_prop(&t, x2, o_bzc(bz));
  *x = t.x; memcpy(p5, t.p, 5 * sizeof(double)); memcpy(c15, t.C, 15 * sizeof(double));
  return rc;
}
int32_t oracle_update(double* p5, double* c15, double ym, double zm, double* chi2) {
  ost t; t.x = 0; memcpy(t.p, p5, 5 * sizeof(double)); memcpy(t.C, c15, 15 * sizeof(double));
  int rc = o_update(&t, ym, zm, chi2);
  memcpy(p5, t.p, 5 * sizeof(double)); memcpy(c15, t.C, 15 * sizeof(double));
  return rc;
}
int32_t oracle_rotate(double* x, double* p5, double* c15, double dalpha) {
  ost t; t.x = *x; memcpy(t.p, p5, 5 * sizeof(double)); memcpy(t.C, c15, 15 * sizeof(double));
  int rc = o_rot(&t, dalpha, o_bzc(0.5));
  *x = t.x; memcpy(p5, t.p, 5 * sizeof(double)); memcpy(c15, t.C, 15 * sizeof(double));
  return rc;
}
int32_t oracle_fit_points(int32_t n, const double* x, const double* y, const double* z, double bz,
                          double* p5, double* c15) {
  ost t;
  o_init_state(&t, x[0], y[0], z[0], p5[2], p5[3], p5[4]);
  if (c15[0] > 0.0) memcpy(t.C, c15, 15 * sizeof(double)); /* caller-given initial covariance */
  double bzc = o_bzc(bz);
  for (int i = 1; i < n; ++i) {
    if (o_prop(&t, x[i], bzc) != 0) return -1;
    if (o_update(&t, y[i], z[i], NULL) != 0) return -1;
  }
  memcpy(p5, t.p, 5 * sizeof(double));
  memcpy(c15, t.C, 15 * sizeof(double));
  return 0;
}

/* ---------------------------------------------------------------- ingest */
static int o_ingest(oracle_result* R, const oracle_input* in) {
  int np[O_NROW];
  for (int r = 0; r < O_NROW; ++r) np[r] = o_npads(r);
  float kz = (float)(1.0 / (0.003125 * in->vdrift));
  for (int64_t i = 0; i < in->n; ++i) {
    int s, r;
    int64_t yu, zu;
    if (in->format == 1) {
      const uint8_t* p = in->packed + 12 * i;
      uint32_t t64; uint16_t pad;
      memcpy(&t64, p, 4); memcpy(&pad, p + 4, 2);
      r = p[8]; s = p[9];
      if (s >= O_NSEC || r >= O_NROW || t64 > 0x3FFFFFFFu) return -1;
      yu = (int64_t)pad - 32 * np[r];
      zu = (int64_t)t64;
    } else {
      s = in->sector[i]; r = in->row[i];
      if (s >= O_NSEC || r >= O_NROW) return -1;
      float yf = in->y[i];
      float zf = in->z ? in->z[i] : in->time[i];
      if (!isfinite(yf) || !isfinite(zf)) return -1;
      float yq = rintf(yf * 160.0f);
      float zq;
      if (in->z) {
        float d = (s < 18) ? (250.0f - zf) : (250.0f + zf);
        zq = rintf(d * kz);
      } else {
        zq = rintf(zf * 320.0f); /* drift time in us -> 1/64 of a 200 ns bin */
      }
      if (fabsf(yq) > 1048576.0f || fabsf(zq) > 1073741824.0f) return -1;
      yu = (int64_t)yq; zu = (int64_t)zq;
    }
    R->yu[i] = (int32_t)yu; R->zu[i] = (int32_t)zu; R->rid[i] = s * O_NROW + r;
  }
  return 0;
}

/* ------------------------------------------------------------ grid + sort */
typedef struct { int32_t rid, cell, orig; } o_key;
static int o_keycmp(const void* a, const void* b) {
  const o_key* x = (const o_key*)a; const o_key* y = (const o_key*)b;
  if (x->rid != y->rid) return x->rid < y->rid ? -1 : 1;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  if (x->orig != y->orig) return x->orig < y->orig ? -1 : 1;
  return 0;
}

static int o_iy(const oracle_result* R, int rid, int64_t yu) {
  int r = rid % O_NROW;
  int64_t half = 32 * (int64_t)o_npads(r);
  int64_t iy = o_floordiv(yu + half, O_CY);
  if (iy < 0) iy = 0;
  if (iy > R->r_ny[rid] - 1) iy = R->r_ny[rid] - 1;
  return (int)iy;
}

static void o_bin(oracle_result* R, uint64_t mask) {
  for (int i = 0; i < O_NROWS; ++i) { R->r_cnt[i] = 0; R->r_zmin[i] = INT32_MAX; R->r_zmax[i] = INT32_MIN; }
  int64_t nsel = 0;
  for (int64_t i = 0; i < R->n; ++i) {
    int s = R->rid[i] / O_NROW;
    if (mask && !((mask >> s) & 1)) continue;
    int rid = R->rid[i];
    R->r_cnt[rid]++;
    if (R->zu[i] < R->r_zmin[rid]) R->r_zmin[rid] = R->zu[i];
    if (R->zu[i] > R->r_zmax[rid]) R->r_zmax[rid] = R->zu[i];
    ++nsel;
  }
  R->nsel = nsel;
  /* grid dimensions */
  R->r_start[0] = 0; R->r_cellbase[0] = 0;
  for (int rid = 0; rid < O_NROWS; ++rid) {
    int r = rid % O_NROW;
    int64_t width = 64 * (int64_t)o_npads(r);
    int64_t ny = (width + O_CY - 1) / O_CY;
    if (ny < 1) ny = 1;
    int64_t n = R->r_cnt[rid];
    int64_t nz = 1, cz = 1;
    if (n > 0) {
      nz = (n + O_T * ny - 1) / (O_T * ny);
      if (nz < 1) nz = 1;
      if (nz > O_NZMAX) nz = O_NZMAX;
      int64_t range = (int64_t)R->r_zmax[rid] - (int64_t)R->r_zmin[rid] + 1;
      cz = (range + nz - 1) / nz;
    } else {
      R->r_zmin[rid] = 0; R->r_zmax[rid] = 0;
    }
    R->r_ny[rid] = (int32_t)ny; R->r_nz[rid] = (int32_t)nz; R->r_cz[rid] = cz;
    R->r_start[rid + 1] = R->r_start[rid] + n;
    R->r_cellbase[rid + 1] = R->r_cellbase[rid] + ny * nz;
  }
  R->ncells = R->r_cellbase[O_NROWS];
  /* keys and sort */
  o_key* K = (o_key*)malloc((size_t)(nsel > 0 ? nsel : 1) * sizeof(o_key));
  int64_t j = 0;
  for (int64_t i = 0; i < R->n; ++i) {
    int rid = R->rid[i];
    if (mask && !((mask >> (rid / O_NROW)) & 1)) continue;
    int64_t iy = o_iy(R, rid, R->yu[i]);
    int64_t iz = (R->zu[i] - (int64_t)R->r_zmin[rid]) / R->r_cz[rid];
    K[j].rid = rid; K[j].cell = (int32_t)(iz * R->r_ny[rid] + iy); K[j].orig = (int32_t)i; ++j;
  }
  qsort(K, (size_t)nsel, sizeof(o_key), o_keycmp);
  R->s_orig = (int32_t*)malloc((size_t)(nsel + 1) * 4); R->s_rid = (int32_t*)malloc((size_t)(nsel + 1) * 4);
  R->s_y = (int32_t*)malloc((size_t)(nsel + 1) * 4); R->s_z = (int32_t*)malloc((size_t)(nsel + 1) * 4);
  R->s_cell = (int32_t*)malloc((size_t)(nsel + 1) * 4);
  for (int64_t i = 0; i < nsel; ++i) {
    R->s_orig[i] = K[i].orig; R->s_rid[i] = K[i].rid; R->s_cell[i] = K[i].cell;
    R->s_y[i] = R->yu[K[i].orig]; R->s_z[i] = R->zu[K[i].orig];
  }
  free(K);
  /* cell starts: cell_start[cellbase[rid] + c] = first sorted index of that cell */
  R->cell_start = (int64_t*)malloc((size_t)(R->ncells + 1) * sizeof(int64_t));
  int64_t h = 0;
  for (int rid = 0; rid < O_NROWS; ++rid) {
    int64_t nc = R->r_cellbase[rid + 1] - R->r_cellbase[rid];
    for (int64_t c = 0; c < nc; ++c) {
      R->cell_start[R->r_cellbase[rid] + c] = h;
      while (h < R->r_start[rid + 1] && R->s_cell[h] == c) ++h;
    }
  }
  R->cell_start[R->ncells] = h;
}

/* Cell rectangle of row rid overlapping [ylo,yhi] x [zlo,zhi] (units).
 * Returns 0 if empty. */
static int o_cellrange(const oracle_result* R, int rid, int64_t ylo, int64_t yhi, int64_t zlo, int64_t zhi,
                       int* iy0, int* iy1, int64_t* iz0, int64_t* iz1) {
  if (R->r_cnt[rid] == 0) return 0;
  *iy0 = o_iy(R, rid, ylo); *iy1 = o_iy(R, rid, yhi);
  int64_t zmin = R->r_zmin[rid], cz = R->r_cz[rid];
  int64_t a = o_floordiv(zlo - zmin, cz), b = o_floordiv(zhi - zmin, cz);
  if (a < 0) a = 0;
  if (b > R->r_nz[rid] - 1) b = R->r_nz[rid] - 1;
  if (a > b) return 0;
  *iz0 = a; *iz1 = b;
  return 1;
}

/* Fit helpers of the tracker: measurement variances follow R->angerr. */
static int o_upd(const oracle_result* R, ost* t, double ym, double zm, double* chi2) {
  double vy, vz;
  o_meas_var(R->angerr, t, &vy, &vz);
  return o_update_v(t, ym, zm, vy, vz, chi2);
}
/* Fresh covariance: the initial diagonal, its (y, zeta) entries the cluster
 * variances at the state's angles. */
static void o_reset_cov(const oracle_result* R, ost* t) {
  memcpy(t->C, O_CINIT, sizeof(O_CINIT));
  o_meas_var(R->angerr, t, &t->C[0], &t->C[2]);
}
static void o_init(const oracle_result* R, ost* t, double x, double y, double z, double s, double tz, double q) {
  o_init_state(t, x, y, z, s, tz, q);
  o_reset_cov(R, t);
}

/* ------------------------------------------------------ NeighboursFinder */
/* Row step 2 (reading, optional): when hit h on row r has no accepted pair
 * on the adjacent rows, it may link across one missing row: up on row r + a,
 * down on row r - b, (a, b) in {(2,1), (1,2), (2,2)}, inside rows 0..151.
 * The straight-line residual generalises to e = (a + b) h - b u - a d (in y
 * and in zeta), whose variance is f = (a + b)^2 + a^2 + b^2 times a cluster's
 * (f = 6 for a = b = 1), so D = 2077 e_y^2 + 1536 e_zeta^2 scaled by 6 / f is
 * the same 2-dof chi2 as before: accepted if 6 D <= 16 * 1536 * 2077 * f;
 * windows a * 1.5 cm, a * 2 cm up and b times those down.  The best pair
 * minimises 6 D / f (compared exactly as D1 f2 < D2 f1), ties to the smaller
 * sorted u, then d. */
static void o_neighbours_gap(const oracle_result* R, int64_t h, int64_t* bu_out, int64_t* bd_out) {
  int rid = R->s_rid[h];
  int r = rid % O_NROW;
  int64_t yh = R->s_y[h], zh = R->s_z[h];
  int64_t bD = -1, bf = 1, bu = -1, bd = -1;
  static const int steps[3][2] = {{2, 1}, {1, 2}, {2, 2}};
  for (int k = 0; k < 3; ++k) {
    int a = steps[k][0], b = steps[k][1];
    if (r + a > O_NROW - 1 || r - b < 0) continue;
    int ru = rid + a, rd = rid - b;
    int uy0, uy1, dy0, dy1; int64_t uz0, uz1, dz0, dz1;
    if (!o_cellrange(R, ru, yh - a * O_WY, yh + a * O_WY, zh - a * O_WZ, zh + a * O_WZ, &uy0, &uy1, &uz0, &uz1)) continue;
    if (!o_cellrange(R, rd, yh - b * O_WY, yh + b * O_WY, zh - b * O_WZ, zh + b * O_WZ, &dy0, &dy1, &dz0, &dz1)) continue;
    int64_t f = (int64_t)(a + b) * (a + b) + a * a + b * b;
    for (int64_t izu = uz0; izu <= uz1; ++izu) {
      int64_t ua = R->cell_start[R->r_cellbase[ru] + izu * R->r_ny[ru] + uy0];
      int64_t ub = R->cell_start[R->r_cellbase[ru] + izu * R->r_ny[ru] + uy1 + 1];
      for (int64_t u = ua; u < ub; ++u) {
        int64_t yu = R->s_y[u], zu = R->s_z[u];
        if (llabs(yu - yh) > a * O_WY || llabs(zu - zh) > a * O_WZ) continue;
        for (int64_t izd = dz0; izd <= dz1; ++izd) {
          int64_t da = R->cell_start[R->r_cellbase[rd] + izd * R->r_ny[rd] + dy0];
          int64_t db = R->cell_start[R->r_cellbase[rd] + izd * R->r_ny[rd] + dy1 + 1];
          for (int64_t d = da; d < db; ++d) {
            int64_t yd = R->s_y[d], zd = R->s_z[d];
            if (llabs(yd - yh) > b * O_WY || llabs(zd - zh) > b * O_WZ) continue;
            int64_t ey = (a + b) * yh - b * yu - a * yd, ez = (a + b) * zh - b * zu - a * zd;
            int64_t D = O_AY * ey * ey + O_AZ * ez * ez;
            if (6 * D > O_DMAX * f) continue;
            int better = bu < 0 || D * bf < bD * f || (D * bf == bD * f && (u < bu || (u == bu && d < bd)));
            if (better) { bD = D; bf = f; bu = u; bd = d; }
          }
        }
      }
    }
  }
  *bu_out = bu; *bd_out = bd;
}

static void o_neighbours(oracle_result* R) {
  int64_t n = R->nsel;
  for (int64_t h = 0; h < n; ++h) { R->up_raw[h] = -1; R->dn_raw[h] = -1; }
  for (int64_t h = 0; h < n; ++h) {
    int rid = R->s_rid[h];
    int r = rid % O_NROW;
    if (r < 1 || r > O_NROW - 2) continue;
    int64_t yh = R->s_y[h], zh = R->s_z[h];
    int ru = rid + 1, rd = rid - 1;
    int uy0 = 0, uy1 = -1, dy0 = 0, dy1 = -1; int64_t uz0 = 0, uz1 = -1, dz0 = 0, dz1 = -1;
    int64_t bestD = INT64_MAX, bu = -1, bd = -1;
    /* an empty cell range on either side leaves no (r+1, r-1) pair */
    if (!o_cellrange(R, ru, yh - O_WY, yh + O_WY, zh - O_WZ, zh + O_WZ, &uy0, &uy1, &uz0, &uz1) ||
        !o_cellrange(R, rd, yh - O_WY, yh + O_WY, zh - O_WZ, zh + O_WZ, &dy0, &dy1, &dz0, &dz1))
      uz1 = uz0 - 1;
    for (int64_t izu = uz0; izu <= uz1; ++izu) {
      int64_t ua = R->cell_start[R->r_cellbase[ru] + izu * R->r_ny[ru] + uy0];
      int64_t ub = R->cell_start[R->r_cellbase[ru] + izu * R->r_ny[ru] + uy1 + 1];
      for (int64_t u = ua; u < ub; ++u) {
        int64_t yu = R->s_y[u], zu = R->s_z[u];
        if (llabs(yu - yh) > O_WY || llabs(zu - zh) > O_WZ) continue;
        for (int64_t izd = dz0; izd <= dz1; ++izd) {
          int64_t da = R->cell_start[R->r_cellbase[rd] + izd * R->r_ny[rd] + dy0];
          int64_t db = R->cell_start[R->r_cellbase[rd] + izd * R->r_ny[rd] + dy1 + 1];
          for (int64_t d = da; d < db; ++d) {
            int64_t yd = R->s_y[d], zd = R->s_z[d];
            if (llabs(yd - yh) > O_WY || llabs(zd - zh) > O_WZ) continue;
            int64_t ey = 2 * yh - yu - yd, ez = 2 * zh - zu - zd;
            int64_t D = O_AY * ey * ey + O_AZ * ez * ez;
            if (D > O_DMAX) continue;
            if (D < bestD || (D == bestD && (u < bu || (u == bu && d < bd)))) { bestD = D; bu = u; bd = d; }
          }
        }
      }
    }
    if (bu < 0 && R->rowstep2) o_neighbours_gap(R, h, &bu, &bd);
    R->up_raw[h] = (int32_t)bu; R->dn_raw[h] = (int32_t)bd;
  }
}

/* ------------------------------------------- NeighboursCleaner + StartHits */
static void o_clean_and_starts(oracle_result* R) {
  int64_t n = R->nsel;
  for (int64_t h = 0; h < n; ++h) {
    int32_t u = R->up_raw[h], d = R->dn_raw[h];
    R->up[h] = (u >= 0 && R->dn_raw[u] == h) ? u : -1;
    R->dn[h] = (d >= 0 && R->up_raw[d] == h) ? d : -1;
  }
  R->nstart = 0;
  R->starts = (int32_t*)malloc((size_t)(n + 1) * 4);
  for (int64_t h = 0; h < n; ++h)
    if (R->dn[h] < 0 && R->up[h] >= 0 && R->up[R->up[h]] >= 0) R->starts[R->nstart++] = (int32_t)h;
}

/* ------------------------------------------------- TrackletConstructor */
static double o_hy(const oracle_result* R, int32_t h) { return (double)R->s_y[h] / 160.0; }
static double o_hz(const oracle_result* R, int32_t h, int32_t zref) { return (double)((int64_t)R->s_z[h] - zref) * R->zunit; }

/* Best hit of row rid inside the +-3 sigma window of the prediction (ties:
 * smaller sorted index); -1 if none passes chi2 <= O_CHI2_FOLLOW. */
static int32_t o_search(const oracle_result* R, int rid, const ost* t, int32_t zref) {
  double vy, vz;
  o_meas_var(R->angerr, t, &vy, &vz);
  double sy2 = t->C[0] + vy, sz2 = t->C[2] + vz;
  double wy = 3.0 * sqrt(sy2), wz = 3.0 * sqrt(sz2);
  int64_t ylo = (int64_t)floor((t->p[0] - wy) * 160.0) - 1, yhi = (int64_t)ceil((t->p[0] + wy) * 160.0) + 1;
  int64_t zlo = zref + (int64_t)floor((t->p[1] - wz) / R->zunit) - 1;
  int64_t zhi = zref + (int64_t)ceil((t->p[1] + wz) / R->zunit) + 1;
  int iy0, iy1; int64_t iz0, iz1;
  if (!o_cellrange(R, rid, ylo, yhi, zlo, zhi, &iy0, &iy1, &iz0, &iz1)) return -1;
  int32_t best = -1; double bchi = 0;
  for (int64_t iz = iz0; iz <= iz1; ++iz) {
    int64_t a = R->cell_start[R->r_cellbase[rid] + iz * R->r_ny[rid] + iy0];
    int64_t b = R->cell_start[R->r_cellbase[rid] + iz * R->r_ny[rid] + iy1 + 1];
    for (int64_t h = a; h < b; ++h) {
      double dy = o_hy(R, (int32_t)h) - t->p[0], dz = o_hz(R, (int32_t)h, zref) - t->p[1];
      if (fabs(dy) > wy || fabs(dz) > wz) continue;
      double chi = dy * dy / sy2 + dz * dz / sz2;
      if (chi > O_CHI2_FOLLOW) continue;
      if (best < 0 || chi < bchi || (chi == bchi && h < best)) { best = (int32_t)h; bchi = chi; }
    }
  }
  return best;
}

static void o_store_state(double* dst, const ost* t) {
  dst[0] = t->x; memcpy(dst + 1, t->p, 5 * sizeof(double)); memcpy(dst + 6, t->C, 15 * sizeof(double));
}
static void o_load_state(ost* t, const double* src) {
  t->x = src[0]; memcpy(t->p, src + 1, 5 * sizeof(double)); memcpy(t->C, src + 6, 15 * sizeof(double));
}

/* Builds tracklet k from start hit h0; hits (ascending rows) to out[], returns count (0: dropped). */
static int o_construct(oracle_result* R, int32_t h0, int32_t* out, double* state, int32_t* zref_out) {
  int32_t chain[O_NROW];
  int nc = 0;
  for (int32_t h = h0; h >= 0 && nc < O_NROW; h = R->up[h]) chain[nc++] = h;
  int32_t zref = R->s_z[h0];
  *zref_out = zref;
  int rid0 = R->s_rid[h0];
  int sbase = rid0 - rid0 % O_NROW;
  double x0 = o_rowx(R->s_rid[chain[0]] % O_NROW), x2 = o_rowx(R->s_rid[chain[2]] % O_NROW);
  double dx = x2 - x0, dy = o_hy(R, chain[2]) - o_hy(R, chain[0]);
  double tphi = dy / dx;
  double s0 = tphi / sqrt(1.0 + tphi * tphi);
  double t0 = (o_hz(R, chain[2], zref) - o_hz(R, chain[0], zref)) / sqrt(dx * dx + dy * dy);
  ost t;
  o_init(R, &t, x0, o_hy(R, chain[0]), o_hz(R, chain[0], zref), s0, t0, 0.0);
  for (int i = 1; i < nc; ++i) {
    int32_t h = chain[i];
    if (o_prop(&t, o_rowx(R->s_rid[h] % O_NROW), R->bzc) != 0) return 0;
    o_upd(R, &t, o_hy(R, h), o_hz(R, h, zref), NULL);
  }
  /* upward following */
  int32_t upl[O_NROW]; int nup = 0;
  ost last = t;
  int32_t top = chain[nc - 1];
  int misses = 0;
  for (int r = R->s_rid[top] % O_NROW + 1; r < O_NROW; ++r) {
    if (o_prop(&t, o_rowx(r), R->bzc) != 0) break;
    if (fabs(t.p[2]) > O_SIN_FOLLOW) break;
    int32_t h = o_search(R, sbase + r, &t, zref);
    if (h >= 0) {
      o_upd(R, &t, o_hy(R, h), o_hz(R, h, zref), NULL);
      upl[nup++] = h; top = h; last = t; misses = 0;
    } else if (++misses >= O_G) break;
  }
  /* downward: restart at the top hit, refit the attached hits, then follow below */
  int32_t att[O_NROW]; int na = 0;
  for (int i = 0; i < nc; ++i) att[na++] = chain[i];
  for (int i = 0; i < nup; ++i) att[na++] = upl[i];
  t = last;
  t.p[0] = o_hy(R, top); t.p[1] = o_hz(R, top, zref);
  o_reset_cov(R, &t);
  for (int i = na - 2; i >= 0; --i) {
    int32_t h = att[i];
    if (o_prop(&t, o_rowx(R->s_rid[h] % O_NROW), R->bzc) != 0) continue;
    o_upd(R, &t, o_hy(R, h), o_hz(R, h, zref), NULL);
  }
  last = t;
  int32_t dnl[O_NROW]; int ndn = 0;
  misses = 0;
  for (int r = R->s_rid[chain[0]] % O_NROW - 1; r >= 0; --r) {
    if (o_prop(&t, o_rowx(r), R->bzc) != 0) break;
    if (fabs(t.p[2]) > O_SIN_FOLLOW) break;
    int32_t h = o_search(R, sbase + r, &t, zref);
    if (h >= 0) {
      o_upd(R, &t, o_hy(R, h), o_hz(R, h, zref), NULL);
      dnl[ndn++] = h; last = t; misses = 0;
    } else if (++misses >= O_G) break;
  }
  int m = 0;
  for (int i = ndn - 1; i >= 0; --i) out[m++] = dnl[i];
  for (int i = 0; i < na; ++i) out[m++] = att[i];
  o_store_state(state, &last);
  return m;
}

static void o_tracklets(oracle_result* R, int reverse) {
  int64_t ns = R->nstart;
  R->tl_nhits = (int32_t*)calloc((size_t)(ns + 1), 4);
  R->tl_kept = (int32_t*)calloc((size_t)(ns + 1), 4);
  R->tl_zref = (int32_t*)calloc((size_t)(ns + 1), 4);
  R->tl_off = (int64_t*)calloc((size_t)(ns + 1), 8);
  R->tl_state = (double*)calloc((size_t)(ns + 1) * 21, 8);
  int32_t* tmp = (int32_t*)malloc((size_t)(ns + 1) * O_NROW * 4);
  for (int64_t q = 0; q < ns; ++q) {
    int64_t k = reverse ? ns - 1 - q : q;
    int m = o_construct(R, R->starts[k], tmp + k * O_NROW, R->tl_state + 21 * k, &R->tl_zref[k]);
    R->tl_nhits[k] = m;
    R->tl_kept[k] = (m >= O_NMIN);
  }
  int64_t tot = 0;
  for (int64_t k = 0; k < ns; ++k) { R->tl_off[k] = tot; tot += R->tl_nhits[k]; }
  R->tl_off[ns] = tot;
  R->tl_nh = tot;
  R->tl_hits = (int32_t*)malloc((size_t)(tot + 1) * 4);
  for (int64_t k = 0; k < ns; ++k) memcpy(R->tl_hits + R->tl_off[k], tmp + k * O_NROW, (size_t)R->tl_nhits[k] * 4);
  free(tmp);
}

/* ----------------------------------------------------- TrackletSelector */
static void o_sector_fit(oracle_result* R, const int32_t* hits, int m, const double* seed_state, int32_t zref,
                         double* st_in, double* st_out) {
  ost sd;
  o_load_state(&sd, seed_state);
  double xa = o_rowx(R->s_rid[hits[0]] % O_NROW);
  ost tmp = sd;
  if (o_prop(&tmp, xa, R->bzc) == 0) sd = tmp;
  ost t;
  o_init(R, &t, xa, o_hy(R, hits[0]), o_hz(R, hits[0], zref), sd.p[2], sd.p[3], sd.p[4]);
  for (int i = 1; i < m; ++i) {
    if (o_prop(&t, o_rowx(R->s_rid[hits[i]] % O_NROW), R->bzc) != 0) continue;
    o_upd(R, &t, o_hy(R, hits[i]), o_hz(R, hits[i], zref), NULL);
  }
  o_store_state(st_out, &t);
  ost u;
  o_init(R, &u, o_rowx(R->s_rid[hits[m - 1]] % O_NROW), o_hy(R, hits[m - 1]), o_hz(R, hits[m - 1], zref),
               t.p[2], t.p[3], t.p[4]);
  for (int i = m - 2; i >= 0; --i) {
    if (o_prop(&u, o_rowx(R->s_rid[hits[i]] % O_NROW), R->bzc) != 0) continue;
    o_upd(R, &u, o_hy(R, hits[i]), o_hz(R, hits[i], zref), NULL);
  }
  o_store_state(st_in, &u);
}

static void o_select(oracle_result* R, int reverse) {
  int64_t ns = R->nstart;
  uint64_t* w = (uint64_t*)calloc((size_t)(R->nsel + 1), 8);
  for (int64_t q = 0; q < ns; ++q) {
    int64_t k = reverse ? ns - 1 - q : q;
    if (!R->tl_kept[k]) continue;
    uint64_t key = ((uint64_t)R->tl_nhits[k] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)k);
    for (int64_t i = R->tl_off[k]; i < R->tl_off[k + 1]; ++i) {
      int32_t h = R->tl_hits[i];
      if (key > w[h]) w[h] = key;
    }
  }
  /* segments: count first */
  int64_t cap = 16, nst = 0, nh = 0, hcap = 1024;
  R->st_sector = (int32_t*)malloc(cap * 4); R->st_tracklet = (int32_t*)malloc(cap * 4);
  R->st_zref = (int32_t*)malloc(cap * 4); R->st_off = (int64_t*)malloc((cap + 1) * 8);
  R->st_in = (double*)malloc(cap * 21 * 8); R->st_out = (double*)malloc(cap * 21 * 8);
  R->st_hits = (int32_t*)malloc(hcap * 4);
  int32_t seg[O_NROW];
  for (int64_t k = 0; k < ns; ++k) {
    if (!R->tl_kept[k]) continue;
    uint64_t key = ((uint64_t)R->tl_nhits[k] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)k);
    int m = 0, prev_row = -1000;
    for (int64_t i = R->tl_off[k]; i <= R->tl_off[k + 1]; ++i) {
      int flush = (i == R->tl_off[k + 1]);
      int32_t h = -1; int row = 0;
      if (!flush) {
        h = R->tl_hits[i];
        if (w[h] != key) continue;
        row = R->s_rid[h] % O_NROW;
        if (m > 0 && row - prev_row - 1 > O_G) flush = 2;
      }
      if (flush) {
        if (m >= O_NMIN) {
          if (nst == cap) {
            cap *= 2;
            R->st_sector = (int32_t*)realloc(R->st_sector, cap * 4); R->st_tracklet = (int32_t*)realloc(R->st_tracklet, cap * 4);
            R->st_zref = (int32_t*)realloc(R->st_zref, cap * 4); R->st_off = (int64_t*)realloc(R->st_off, (cap + 1) * 8);
            R->st_in = (double*)realloc(R->st_in, cap * 21 * 8); R->st_out = (double*)realloc(R->st_out, cap * 21 * 8);
          }
          while (nh + m > hcap) { hcap *= 2; R->st_hits = (int32_t*)realloc(R->st_hits, hcap * 4); }
          R->st_sector[nst] = R->s_rid[seg[0]] / O_NROW;
          R->st_tracklet[nst] = (int32_t)k;
          R->st_zref[nst] = R->s_z[seg[0]];
          R->st_off[nst] = nh;
          memcpy(R->st_hits + nh, seg, (size_t)m * 4);
          o_sector_fit(R, seg, m, R->tl_state + 21 * k, R->st_zref[nst], R->st_in + 21 * nst, R->st_out + 21 * nst);
          nh += m; ++nst;
        }
        m = 0;
        if (flush == 1) break;
      }
      seg[m++] = h; prev_row = row;
    }
  }
  R->st_off[nst] = nh;
  R->nst = nst; R->st_nh = nh;
  free(w);
}

/* --------------------------------------------------------------- Merger */
typedef struct { double chi2; int32_t a, b; } o_pair;
static int o_paircmp(const void* x, const void* y) {
  const o_pair* p = (const o_pair*)x; const o_pair* q = (const o_pair*)y;
  if (p->chi2 != q->chi2) return p->chi2 < q->chi2 ? -1 : 1;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

/* chi2 = d^T M^{-1} d for a symmetric positive-definite 5x5 M (Cholesky). */
static int o_chi2_5(const double* d, const double* c15, double* chi2) {
  double L[5][5];
  memset(L, 0, sizeof(L));
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = c15[o_ix(i, j)];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) { if (!(s > 0)) return -1; L[i][i] = sqrt(s); }
      else L[i][j] = s / L[j][j];
    }
  }
  double v[5];
  for (int i = 0; i < 5; ++i) { double s = d[i]; for (int k = 0; k < i; ++k) s -= L[i][k] * v[k]; v[i] = s / L[i][i]; }
  double c = 0;
  for (int i = 0; i < 5; ++i) c += v[i] * v[i];
  *chi2 = c;
  return 0;
}

static void o_merge(oracle_result* R, uint64_t mask) {
  int64_t nst = R->nst;
  R->st_next = (int32_t*)malloc((size_t)(nst + 1) * 4);
  R->st_prev = (int32_t*)malloc((size_t)(nst + 1) * 4);
  for (int64_t i = 0; i < nst; ++i) { R->st_next[i] = -1; R->st_prev[i] = -1; }
  double tn = o_tan10();
  int8_t* near_out = (int8_t*)calloc((size_t)(nst + 1), 1);
  int8_t* near_in = (int8_t*)calloc((size_t)(nst + 1), 1);
  for (int64_t i = 0; i < nst; ++i) {
    const double* so = R->st_out + 21 * i; const double* si = R->st_in + 21 * i;
    if (fabs(so[1]) >= so[0] * tn - O_EDGE) near_out[i] = so[1] > 0 ? 1 : -1;
    if (fabs(si[1]) >= si[0] * tn - O_EDGE) near_in[i] = si[1] > 0 ? 1 : -1;
  }
  int64_t pcap = 1024, npair = 0;
  R->pair_ab = (int32_t*)malloc(pcap * 2 * 4); R->pair_chi2 = (double*)malloc(pcap * 8);
  o_pair* P = (o_pair*)malloc(sizeof(o_pair) * 1024);
  int64_t Pcap = 1024;
  for (int side = 0; side < 2; ++side)
    for (int j = 0; j < 18; ++j)
      for (int d = 1; d >= -1; d -= 2) {
        int s = side * 18 + j, s2 = side * 18 + (j + d + 18) % 18;
        if (mask && (!((mask >> s) & 1) || !((mask >> s2) & 1))) continue;
        int64_t np = 0;
        for (int64_t a = 0; a < nst; ++a) {
          if (R->st_sector[a] != s || near_out[a] != d) continue;
          for (int64_t b = 0; b < nst; ++b) {
            if (R->st_sector[b] != s2 || near_in[b] != -d) continue;
            const double* A = R->st_out + 21 * a; const double* B = R->st_in + 21 * b;
            double dzr = (double)((int64_t)R->st_zref[a] - R->st_zref[b]) * R->zunit;
            if (fabs(dzr + A[2] - B[2]) > O_DZETA_PRE) continue;
            ost t; o_load_state(&t, A);
            if (o_rot(&t, d * 20.0 * O_PI / 180.0, R->bzc) != 0) continue;
            if (o_prop(&t, B[0], R->bzc) != 0) continue;
            double dv[5], cs[15];
            for (int q = 0; q < 5; ++q) dv[q] = t.p[q] - B[1 + q];
            dv[1] += dzr;
            for (int q = 0; q < 15; ++q) cs[q] = t.C[q] + B[6 + q];
            double chi2;
            if (o_chi2_5(dv, cs, &chi2) != 0) continue;
            if (!(chi2 <= O_CHI2_MERGE)) continue;
            if (np == Pcap) { Pcap *= 2; P = (o_pair*)realloc(P, sizeof(o_pair) * Pcap); }
            P[np].chi2 = chi2; P[np].a = (int32_t)a; P[np].b = (int32_t)b; ++np;
          }
        }
        qsort(P, (size_t)np, sizeof(o_pair), o_paircmp);
        for (int64_t q = 0; q < np; ++q) {
          if (npair == pcap) { pcap *= 2; R->pair_ab = (int32_t*)realloc(R->pair_ab, pcap * 2 * 4); R->pair_chi2 = (double*)realloc(R->pair_chi2, pcap * 8); }
          R->pair_ab[2 * npair] = P[q].a; R->pair_ab[2 * npair + 1] = P[q].b; R->pair_chi2[npair] = P[q].chi2; ++npair;
          if (R->st_next[P[q].a] >= 0 || R->st_prev[P[q].b] >= 0) continue;
          R->st_next[P[q].a] = P[q].b; R->st_prev[P[q].b] = P[q].a;
        }
      }
  R->npair = npair;
  free(P); free(near_out); free(near_in);
  /* cycles: a track on a closed loop of links has a predecessor; cut the loop
   * at its smallest id, which becomes a head */
  int8_t* seen = (int8_t*)calloc((size_t)(nst + 1), 1);
  for (int64_t i = 0; i < nst; ++i) if (R->st_prev[i] < 0) for (int64_t c = i; c >= 0; c = R->st_next[c]) seen[c] = 1;
  for (int64_t i = 0; i < nst; ++i) {
    if (seen[i]) continue;
    int64_t c = i;  /* i is the smallest unseen id of its loop */
    R->st_next[R->st_prev[i]] = -1;
    R->st_prev[i] = -1;
    for (; c >= 0; c = R->st_next[c]) seen[c] = 1;
  }
  free(seen);
}

/* ----------------------------------------------------------- final refit */
static void o_final(oracle_result* R) {
  int64_t nst = R->nst;
  int64_t nt = 0;
  for (int64_t i = 0; i < nst; ++i) if (R->st_prev[i] < 0) ++nt;
  R->ntrk = nt;
  int64_t n1 = nt + 1;
  R->trk_off = (int64_t*)calloc((size_t)n1, 8); R->trk_cl = (int32_t*)malloc((size_t)(R->st_nh + 1) * 4);
  R->trk_x = (double*)calloc((size_t)n1, 8); R->trk_alpha = (double*)calloc((size_t)n1, 8);
  R->trk_par = (double*)calloc((size_t)n1 * 5, 8); R->trk_cov = (double*)calloc((size_t)n1 * 15, 8);
  R->trk_chi2 = (double*)calloc((size_t)n1, 8);
  R->trk_ndf = (int32_t*)calloc((size_t)n1, 4); R->trk_sector = (int32_t*)calloc((size_t)n1, 4);
  R->trk_flags = (int32_t*)calloc((size_t)n1, 4); R->trk_zref = (int32_t*)calloc((size_t)n1, 4);
  R->trk_head = (int32_t*)calloc((size_t)n1, 4); R->trk_nseg = (int32_t*)calloc((size_t)n1, 4);
  int32_t* hs = (int32_t*)malloc((size_t)(R->st_nh + 1) * 4);
  int32_t* hsec = (int32_t*)malloc((size_t)(R->st_nh + 1) * 4);
  int64_t o = 0, it = 0;
  for (int64_t head = 0; head < nst; ++head) {
    if (R->st_prev[head] >= 0) continue;
    int64_t m = 0, tail = head;
    int nseg = 0;
    for (int64_t c = head; c >= 0; c = R->st_next[c]) {
      for (int64_t i = R->st_off[c]; i < R->st_off[c + 1]; ++i) { hs[m] = R->st_hits[i]; hsec[m] = R->st_sector[c]; ++m; }
      tail = c; ++nseg;
    }
    int32_t zref = R->s_z[hs[0]];
    const double* so = R->st_out + 21 * tail;
    int frame = hsec[m - 1];
    ost t;
    o_init(R, &t, o_rowx(R->s_rid[hs[m - 1]] % O_NROW), o_hy(R, hs[m - 1]), o_hz(R, hs[m - 1], zref), so[3], so[4], so[5]);
    double chi2 = 0; int used = 1; int flags = nseg > 1 ? 2 : 0;
    for (int64_t i = m - 2; i >= 0; --i) {
      int32_t h = hs[i];
      if (hsec[i] != frame) {
        if (o_rot(&t, o_alpha(hsec[i]) - o_alpha(frame), R->bzc) != 0) { flags |= 4; break; }
        frame = hsec[i];
      }
      if (o_prop(&t, o_rowx(R->s_rid[h] % O_NROW), R->bzc) != 0) continue;
      double c2;
      if (o_upd(R, &t, o_hy(R, h), o_hz(R, h, zref), &c2) != 0) continue;
      chi2 += c2; ++used;
    }
    R->trk_off[it] = o;
    for (int64_t i = 0; i < m; ++i) R->trk_cl[o + i] = R->s_orig[hs[i]];
    o += m;
    int side = o_side(frame);
    double sg = (side > 0) ? -1.0 : 1.0; /* tan(lambda) = dz/ds = -side * dzeta/ds */
    R->trk_x[it] = t.x; R->trk_alpha[it] = o_alpha(frame);
    double* par = R->trk_par + 5 * it; double* cov = R->trk_cov + 15 * it;
    memcpy(par, t.p, 5 * sizeof(double)); memcpy(cov, t.C, 15 * sizeof(double));
    par[3] *= sg;
    for (int i = 0; i < 5; ++i) if (i != 3) cov[o_ix(3, i)] *= sg;
    R->trk_chi2[it] = chi2; R->trk_ndf[it] = 2 * used - 5; R->trk_sector[it] = frame;
    R->trk_flags[it] = flags; R->trk_zref[it] = zref;
    R->trk_head[it] = (int32_t)head; R->trk_nseg[it] = nseg;
    ++it;
  }
  R->trk_off[nt] = o; R->trk_ncl = o;
  free(hs); free(hsec);
}

/* ------------------------------------------- continuous-readout completion
 * Sec. 2: with continuous readout the drift coordinate of a cluster is
 * v_d (t0 + t_drift), so a track's own clusters fix its collision time t0
 * only up to the unknown z of its vertex, and tracks are assigned to
 * collisions after tracking.  The paper gives no method; the readings here
 * (all constants below are ours):
 *  - t0 bounds from the clusters: every cluster lies at 0 <= |z| <= 250 cm,
 *    so zeta_max - 250 <= v_d t0 <= zeta_min; zeta is linear along the
 *    helix, so its extremes are those of the track's two end clusters;
 *  - vertex t0: the track extrapolated to its closest approach to the beam
 *    axis in the transverse plane, assuming z_vertex = 0 there, clamped into
 *    the bounds; its error adds the beam-spot length O_SIGMA_ZV;
 *  - membrane crossing: a track segment that runs towards the central
 *    membrane (z = 0) and ends, and a segment of the other side (in the
 *    same sector angle or a neighbouring one) that starts a few rows further
 *    out, are the two halves of
 *    one track when their y, sin(phi), tan(lambda), q/pT agree (chi2 on 4
 *    parameters) at the outer segment's first cluster.  z is continuous at
 *    the crossing, so at any common x the membrane sits at the mean of the
 *    two segments' drift coordinates, which gives t0 without any assumption
 *    on the vertex; one partner per segment, greedy in (chi2, inner, outer);
 *  - collision assignment: among the interaction times of the TF (input,
 *    sorted ascending) compatible with the t0 bounds (plus O_T0_SLACK), the
 *    one nearest to the track's t0 (ties: the earlier).                   */
#define O_SIGMA_ZV 5.0       /* beam-spot length, cm                          */
#define O_MEM_ROWGAP 10      /* outer segment starts 1..10 rows further out   */
#define O_MEM_DZU 384        /* |zeta_out(inner) - zeta_in(outer)|, units      */
#define O_CHI2_MEM 25.0      /* chi2 on 4 parameters                           */
#define O_MEM_ZTOL 1.0       /* membrane zeta may sit this far below a cluster */
#define O_T0_SLACK 0.3       /* us, on the t0 bounds when assigning            */

/* Signed transverse arc length from (x0, y0, direction phi0) to the point of
 * the circle of curvature k (dphi/ds) closest to the origin: with
 * t = -(x0 cos + y0 sin) and d = x0 sin - y0 cos, the turning angle to that
 * point is atan2(k t, 1 - k d), which tends to the straight line's t. */
static double o_dca_arc(double x0, double y0, double snp, double k) {
  double csp = sqrt((1.0 - snp) * (1.0 + snp));
  double t = -(x0 * csp + y0 * snp), d = x0 * snp - y0 * csp;
  if (k == 0.0) return t;
  return atan2(k * t, 1.0 - k * d) / k;
}

double oracle_dca_arc(double x0, double y0, double snp, double k) { return o_dca_arc(x0, y0, snp, k); }

typedef struct { int32_t zmin, zmax, zin, zout, rin, rout, sin, sout; } o_ends;

static void o_continuous(oracle_result* R, const oracle_input* in) {
  int64_t nt = R->ntrk, n1 = nt + 1;
  double zu = R->zunit, vd = in->vdrift;
  R->trk_t0 = (double*)calloc((size_t)n1, 8); R->trk_t0err = (double*)calloc((size_t)n1, 8);
  R->trk_t0lo = (double*)calloc((size_t)n1, 8); R->trk_t0hi = (double*)calloc((size_t)n1, 8);
  R->trk_mate = (int32_t*)malloc((size_t)n1 * 4); R->trk_coll = (int32_t*)malloc((size_t)n1 * 4);
  o_ends* E = (o_ends*)calloc((size_t)n1, sizeof(o_ends));
  for (int64_t i = 0; i < nt; ++i) {
    o_ends* e = E + i;
    int32_t c0 = R->trk_cl[R->trk_off[i]], c1 = R->trk_cl[R->trk_off[i + 1] - 1];
    e->zin = R->zu[c0]; e->zout = R->zu[c1];
    e->rin = R->rid[c0] % O_NROW; e->sin = R->rid[c0] / O_NROW;
    e->rout = R->rid[c1] % O_NROW; e->sout = R->rid[c1] / O_NROW;
    /* zeta is linear along the helix: its extremes sit at the end clusters */
    e->zmin = e->zin < e->zout ? e->zin : e->zout;
    e->zmax = e->zin < e->zout ? e->zout : e->zin;
    R->trk_t0lo[i] = ((double)e->zmax * zu - 250.0) / vd;
    R->trk_t0hi[i] = (double)e->zmin * zu / vd;
    R->trk_mate[i] = -1;
  }
  /* membrane pairs: inner segment a (towards the membrane), outer b */
  int64_t np = 0, pcap = 256;
  o_pair* P = (o_pair*)malloc(sizeof(o_pair) * pcap);
  double* zmid = NULL; /* membrane zeta (cm, absolute) and its variance per pair */
  double* zvar = NULL;
  zmid = (double*)malloc(sizeof(double) * pcap); zvar = (double*)malloc(sizeof(double) * pcap);
  /* tracks by the sector of their first cluster, ascending ids */
  int64_t bstart[37] = {0};
  for (int64_t i = 0; i < nt; ++i) bstart[E[i].sin + 1]++;
  for (int q = 0; q < 36; ++q) bstart[q + 1] += bstart[q];
  int64_t* bfill = (int64_t*)calloc(36, sizeof(int64_t));
  int32_t* bsec = (int32_t*)malloc(sizeof(int32_t) * n1);
  for (int64_t i = 0; i < nt; ++i) bsec[bstart[E[i].sin] + bfill[E[i].sin]++] = (int32_t)i;
  free(bfill);
  for (int64_t a = 0; a < nt; ++a) {
    const o_ends* ea = E + a;
    const double* pa = R->trk_par + 5 * a;
    int sa = o_side(ea->sout);
    if ((R->trk_flags[a] & 4) || R->trk_sector[a] != ea->sin) continue;
    if (ea->rout > O_NROW - 2 || !(sa * pa[3] < 0.0)) continue;
    for (int d = -1; d <= 1; ++d) {
      /* the outer piece may start one sector angle off the inner piece's end */
      int jb = (ea->sout % 18 + d + 18) % 18;
      int sb_need = (sa > 0 ? 18 : 0) + jb;
      int jrot = ((jb - ea->sin % 18) % 18 + 27) % 18 - 9; /* in [-9, 8] */
      if (jrot < -2 || jrot > 2) continue;
      for (int64_t qb = bstart[sb_need]; qb < bstart[sb_need + 1]; ++qb) {
        int64_t b = bsec[qb];
        const o_ends* eb = E + b;
        const double* pb = R->trk_par + 5 * b;
        if ((R->trk_flags[b] & 4) || R->trk_sector[b] != eb->sin) continue;
        if (eb->rin < 1 || !(o_side(eb->sin) * pb[3] > 0.0)) continue;
        int gap = eb->rin - ea->rout;
        if (gap < 1 || gap > O_MEM_ROWGAP) continue;
        if (abs(eb->zin - ea->zout) > O_MEM_DZU) continue;
        /* a's state in the tracker's convention (dzeta/ds), turned into b's
         * frame and moved to b's x */
        ost t;
        double sga = (sa > 0) ? -1.0 : 1.0;
        t.x = R->trk_x[a];
        memcpy(t.p, pa, 5 * sizeof(double)); memcpy(t.C, R->trk_cov + 15 * a, 15 * sizeof(double));
        t.p[3] *= sga;
        for (int q = 0; q < 5; ++q) if (q != 3) t.C[o_ix(3, q)] *= sga;
        if (jrot != 0 && o_rot(&t, jrot * 20.0 * O_PI / 180.0, R->bzc) != 0) continue;
        if (o_prop(&t, R->trk_x[b], R->bzc) != 0) continue;
        t.p[3] *= sga;
        for (int q = 0; q < 5; ++q) if (q != 3) t.C[o_ix(3, q)] *= sga;
        static const int idx[4] = {0, 2, 3, 4};
        double dv[5] = {0}, cs[15] = {0};
        const double* cb = R->trk_cov + 15 * b;
        for (int i = 0; i < 4; ++i) {
          dv[i] = t.p[idx[i]] - pb[idx[i]];
          for (int j = 0; j <= i; ++j) cs[o_ix(i, j)] = t.C[o_ix(idx[i], idx[j])] + cb[o_ix(idx[i], idx[j])];
        }
        cs[o_ix(4, 4)] = 1.0; /* 4x4 block padded with a unit pivot: dv[4] = 0 adds nothing */
        double chi2;
        if (o_chi2_5(dv, cs, &chi2) != 0 || !(chi2 <= O_CHI2_MEM)) continue;
        double za = (double)R->trk_zref[a] * zu + t.p[1];
        double zb = (double)R->trk_zref[b] * zu + pb[1];
        double zm = 0.5 * (za + zb);
        int32_t zmx = ea->zmax > eb->zmax ? ea->zmax : eb->zmax;
        if (zm < (double)zmx * zu - O_MEM_ZTOL) continue;
        if (np == pcap) {
          pcap *= 2;
          P = (o_pair*)realloc(P, sizeof(o_pair) * pcap);
          zmid = (double*)realloc(zmid, sizeof(double) * pcap); zvar = (double*)realloc(zvar, sizeof(double) * pcap);
        }
        P[np].chi2 = chi2; P[np].a = (int32_t)a; P[np].b = (int32_t)b;
        zmid[np] = zm; zvar[np] = 0.25 * (t.C[o_ix(1, 1)] + cb[o_ix(1, 1)]);
        ++np;
      }
    }
  }
  free(bsec);
  /* greedy over pairs sorted by (chi2, a, b); the membrane zeta of a taken
   * pair is found again by its (a, b) after sorting */
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (np + 1));
  o_pair* S = (o_pair*)malloc(sizeof(o_pair) * (np + 1));
  memcpy(S, P, sizeof(o_pair) * np);
  qsort(S, (size_t)np, sizeof(o_pair), o_paircmp);
  for (int64_t q = 0; q < np; ++q) {
    int64_t k = 0;
    while (!(P[k].a == S[q].a && P[k].b == S[q].b)) ++k;
    order[q] = k;
  }
  int32_t* tm = (int32_t*)calloc((size_t)n1, 4); /* 1: t0 from the membrane */
  for (int64_t q = 0; q < np; ++q) {
    int32_t a = S[q].a, b = S[q].b;
    if (R->trk_mate[a] >= 0 || R->trk_mate[b] >= 0) continue;
    R->trk_mate[a] = b; R->trk_mate[b] = a;
    double t0 = (zmid[order[q]] - 250.0) / vd, er = sqrt(zvar[order[q]]) / vd;
    double lo = R->trk_t0lo[a] > R->trk_t0lo[b] ? R->trk_t0lo[a] : R->trk_t0lo[b];
    double hi = R->trk_t0hi[a] < R->trk_t0hi[b] ? R->trk_t0hi[a] : R->trk_t0hi[b];
    R->trk_t0[a] = R->trk_t0[b] = t0; R->trk_t0err[a] = R->trk_t0err[b] = er;
    R->trk_t0lo[a] = R->trk_t0lo[b] = lo; R->trk_t0hi[a] = R->trk_t0hi[b] = hi;
    tm[a] = tm[b] = 1;
    R->trk_flags[a] |= 8; R->trk_flags[b] |= 8;
  }
  R->nmpair = np;
  R->mpair_ab = (int32_t*)malloc(sizeof(int32_t) * 2 * (np + 1)); R->mpair_chi2 = (double*)malloc(sizeof(double) * (np + 1));
  for (int64_t q = 0; q < np; ++q) { R->mpair_ab[2 * q] = S[q].a; R->mpair_ab[2 * q + 1] = S[q].b; R->mpair_chi2[q] = S[q].chi2; }
  free(P); free(S); free(order); free(zmid); free(zvar);
  /* vertex t0 of the tracks without a partner */
  for (int64_t i = 0; i < nt; ++i) {
    if (tm[i]) continue;
    const double* p = R->trk_par + 5 * i; const double* C = R->trk_cov + 15 * i;
    int side = o_side(R->trk_sector[i]);
    double lo = R->trk_t0lo[i], hi = R->trk_t0hi[i];
    if (!(fabs(p[2]) < 1.0)) { /* no direction: the middle of the bounds */
      R->trk_t0[i] = 0.5 * (lo + hi); R->trk_t0err[i] = 0.5 * (hi - lo);
      continue;
    }
    double k = p[4] * R->bzc;
    double s = o_dca_arc(R->trk_x[i], p[0], p[2], k);
    double dzds = -(double)side * p[3]; /* dzeta/ds */
    double zv = (double)R->trk_zref[i] * zu + p[1] + dzds * s;
    double t0 = (zv - 250.0) / vd;
    if (t0 < lo) t0 = lo;
    if (t0 > hi) t0 = hi;
    /* variance of zeta + s dzeta/ds (s held fixed) plus the beam spot */
    double c13 = -(double)side * C[o_ix(1, 3)], c33 = C[o_ix(3, 3)];
    double var = C[o_ix(1, 1)] + 2.0 * s * c13 + s * s * c33;
    if (!(var >= 0.0)) var = 0.0;
    var += O_SIGMA_ZV * O_SIGMA_ZV;
    R->trk_t0[i] = t0; R->trk_t0err[i] = sqrt(var) / vd;
  }
  free(tm);
  /* collision assignment */
  for (int64_t i = 0; i < nt; ++i) {
    int32_t best = -1; double bd = 0;
    for (int64_t c = 0; c < in->n_coll; ++c) {
      double tc = in->coll_time[c];
      if (tc < R->trk_t0lo[i] - O_T0_SLACK || tc > R->trk_t0hi[i] + O_T0_SLACK) continue;
      double d = fabs(tc - R->trk_t0[i]);
      if (best < 0 || d < bd) { best = (int32_t)c; bd = d; }
    }
    R->trk_coll[i] = best;
  }
  free(E);
}

/* ---------------------------------------------------------------- driver */
static void o_add(oracle_result* R, const char* name, const void* p, int64_t n, int32_t type) {
  R->fields[R->nf].name = name; R->fields[R->nf].ptr = p; R->fields[R->nf].n = n; R->fields[R->nf].type = type; R->nf++;
}

oracle_result* oracle_run(const oracle_input* in, int32_t* status) {
  oracle_result* R = (oracle_result*)calloc(1, sizeof(oracle_result));
  R->n = in->n;
  R->zunit = 0.003125 * in->vdrift;
  R->bzc = o_bzc(in->bz);
  R->angerr = in->angular_errors != 0;
  R->rowstep2 = in->row_step2 != 0;
  int64_t n1 = in->n + 1;
  R->yu = (int32_t*)malloc((size_t)n1 * 4); R->zu = (int32_t*)malloc((size_t)n1 * 4); R->rid = (int32_t*)malloc((size_t)n1 * 4);
  if (o_ingest(R, in) != 0) { *status = -1; oracle_free(R); return NULL; }
  o_bin(R, in->sector_mask);
  int64_t m1 = R->nsel + 1;
  R->up_raw = (int32_t*)malloc((size_t)m1 * 4); R->dn_raw = (int32_t*)malloc((size_t)m1 * 4);
  R->up = (int32_t*)malloc((size_t)m1 * 4); R->dn = (int32_t*)malloc((size_t)m1 * 4);
  o_neighbours(R);
  o_clean_and_starts(R);
  o_tracklets(R, in->reverse_tracklet_order);
  o_select(R, in->reverse_tracklet_order);
  o_merge(R, in->sector_mask);
  o_final(R);
  o_continuous(R, in);
  if (in->compress) {
    int64_t n = R->n;
    int32_t* sec = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t* row = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    double* qpt = (double*)malloc(sizeof(double) * ((size_t)R->ntrk + 1));
    for (int64_t i = 0; i < n; ++i) { sec[i] = R->rid[i] / O_NROW; row[i] = R->rid[i] % O_NROW; }
    for (int64_t t = 0; t < R->ntrk; ++t) qpt[t] = R->trk_par[5 * t + 4];
    R->ctf_bytes = oracle_ctf_encode(n, sec, row, R->yu, R->zu, R->ntrk, R->trk_off, R->trk_cl, qpt, R->s_orig,
                                     R->nsel, &R->ctf);
    free(sec); free(row); free(qpt);
  }
  o_add(R, "yu", R->yu, R->n, 0); o_add(R, "zu", R->zu, R->n, 0); o_add(R, "rid", R->rid, R->n, 0);
  o_add(R, "sorted_orig", R->s_orig, R->nsel, 0); o_add(R, "sorted_rid", R->s_rid, R->nsel, 0);
  o_add(R, "sorted_y", R->s_y, R->nsel, 0); o_add(R, "sorted_z", R->s_z, R->nsel, 0); o_add(R, "sorted_cell", R->s_cell, R->nsel, 0);
  o_add(R, "row_count", R->r_cnt, O_NROWS, 0); o_add(R, "row_zmin", R->r_zmin, O_NROWS, 0); o_add(R, "row_zmax", R->r_zmax, O_NROWS, 0);
  o_add(R, "row_ny", R->r_ny, O_NROWS, 0); o_add(R, "row_nz", R->r_nz, O_NROWS, 0); o_add(R, "row_cz", R->r_cz, O_NROWS, 1);
  o_add(R, "row_start", R->r_start, O_NROWS + 1, 1); o_add(R, "row_cellbase", R->r_cellbase, O_NROWS + 1, 1);
  o_add(R, "cell_start", R->cell_start, R->ncells + 1, 1);
  o_add(R, "up_raw", R->up_raw, R->nsel, 0); o_add(R, "dn_raw", R->dn_raw, R->nsel, 0);
  o_add(R, "up", R->up, R->nsel, 0); o_add(R, "dn", R->dn, R->nsel, 0);
  o_add(R, "starts", R->starts, R->nstart, 0);
  o_add(R, "tl_nhits", R->tl_nhits, R->nstart, 0); o_add(R, "tl_kept", R->tl_kept, R->nstart, 0);
  o_add(R, "tl_zref", R->tl_zref, R->nstart, 0); o_add(R, "tl_off", R->tl_off, R->nstart + 1, 1);
  o_add(R, "tl_hits", R->tl_hits, R->tl_nh, 0); o_add(R, "tl_state", R->tl_state, R->nstart * 21, 2);
  o_add(R, "st_sector", R->st_sector, R->nst, 0); o_add(R, "st_tracklet", R->st_tracklet, R->nst, 0);
  o_add(R, "st_zref", R->st_zref, R->nst, 0); o_add(R, "st_off", R->st_off, R->nst + 1, 1);
  o_add(R, "st_hits", R->st_hits, R->st_nh, 0); o_add(R, "st_in", R->st_in, R->nst * 21, 2);
  o_add(R, "st_out", R->st_out, R->nst * 21, 2); o_add(R, "st_next", R->st_next, R->nst, 0);
  o_add(R, "st_prev", R->st_prev, R->nst, 0);
  o_add(R, "pair_ab", R->pair_ab, R->npair * 2, 0); o_add(R, "pair_chi2", R->pair_chi2, R->npair, 2);
  o_add(R, "trk_off", R->trk_off, R->ntrk + 1, 1); o_add(R, "trk_cl", R->trk_cl, R->trk_ncl, 0);
  o_add(R, "trk_x", R->trk_x, R->ntrk, 2); o_add(R, "trk_alpha", R->trk_alpha, R->ntrk, 2);
  o_add(R, "trk_par", R->trk_par, R->ntrk * 5, 2); o_add(R, "trk_cov", R->trk_cov, R->ntrk * 15, 2);
  o_add(R, "trk_chi2", R->trk_chi2, R->ntrk, 2); o_add(R, "trk_ndf", R->trk_ndf, R->ntrk, 0);
  o_add(R, "trk_sector", R->trk_sector, R->ntrk, 0); o_add(R, "trk_flags", R->trk_flags, R->ntrk, 0);
  o_add(R, "trk_zref", R->trk_zref, R->ntrk, 0); o_add(R, "trk_head", R->trk_head, R->ntrk, 0);
  o_add(R, "trk_nseg", R->trk_nseg, R->ntrk, 0);
  o_add(R, "trk_t0", R->trk_t0, R->ntrk, 2); o_add(R, "trk_t0err", R->trk_t0err, R->ntrk, 2);
  o_add(R, "trk_t0lo", R->trk_t0lo, R->ntrk, 2); o_add(R, "trk_t0hi", R->trk_t0hi, R->ntrk, 2);
  o_add(R, "trk_mate", R->trk_mate, R->ntrk, 0); o_add(R, "trk_coll", R->trk_coll, R->ntrk, 0);
  o_add(R, "mpair_ab", R->mpair_ab, R->nmpair * 2, 0); o_add(R, "mpair_chi2", R->mpair_chi2, R->nmpair, 2);
  o_add(R, "ctf", R->ctf, R->ctf_bytes, 3);
  *status = 0;
  return R;
}

int64_t oracle_get(oracle_result* R, const char* name, const void** ptr, int32_t* type) {
  for (int i = 0; i < R->nf; ++i)
    if (strcmp(R->fields[i].name, name) == 0) { *ptr = R->fields[i].ptr; *type = R->fields[i].type; return R->fields[i].n; }
  return -1;
}

void oracle_free(oracle_result* R) {
  if (!R) return;
  void* ps[] = {R->yu, R->zu, R->rid, R->s_orig, R->s_rid, R->s_y, R->s_z, R->s_cell, R->cell_start,
                R->up_raw, R->dn_raw, R->up, R->dn, R->starts, R->tl_nhits, R->tl_kept, R->tl_zref, R->tl_off,
                R->tl_hits, R->tl_state, R->st_sector, R->st_tracklet, R->st_zref, R->st_off, R->st_hits,
                R->st_in, R->st_out, R->st_next, R->st_prev, R->pair_ab, R->pair_chi2, R->trk_off, R->trk_cl,
                R->trk_x, R->trk_alpha, R->trk_par, R->trk_cov, R->trk_chi2, R->trk_ndf, R->trk_sector,
                R->trk_flags, R->trk_zref, R->trk_head, R->trk_nseg, R->trk_t0, R->trk_t0err, R->trk_t0lo,
                R->trk_t0hi, R->trk_mate, R->trk_coll, R->mpair_ab, R->mpair_chi2, R->ctf};
  for (size_t i = 0; i < sizeof(ps) / sizeof(ps[0]); ++i) free(ps[i]);
  free(R);
}
