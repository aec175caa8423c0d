/*
 * o2gen.c - seeded synthetic TPC Time-Frame generator.
 *
 * Stands in for the ALICE Time Frames that the paper feeds to its standalone
 * benchmark (Sec. 3.2, "Standalone benchmark"): Pb-Pb-like collisions in
 * continuous readout (Sec. 2, the Time Frame of 128 orbits), where the drift
 * time of every cluster maps linearly onto the beam coordinate and collisions
 * overlap in time.
 *
 * This module is shared input plumbing: it holds detector simulation only
 * (helix geometry, pad-row crossings, smearing, noise, packing into the
 * cluster formats) and none of the tracker's arithmetic.  Random numbers come
 * from a counter-based generator (splitmix64 finaliser applied to
 * key + counter * golden-ratio increment), so the output does not depend on
 * the number of threads.
 *
 * Geometry (the detector description both the tracker and this generator
 * assume): 36 sectors (0-17 on side A, z > 0; 18-35 on side C), sector s
 * centred at azimuth ((s mod 18) * 20 + 10) degrees, 152 pad-row planes at
 * local x_r = 85 + r * 160/151 cm, pad pitch 0.4 cm, nPads(r) =
 * floor(2 x_r tan(10 deg) / 0.4), drift length 250 cm.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define G_NROW 152
#define G_NSEC 36
#define G_DRIFT_LEN 250.0
#define G_PI 3.14159265358979323846
#define G_RHO_MAX 250.0 /* cm, beyond the outermost pad-row corner */

/* ---------------------------------------------------------------- RNG */
static inline uint64_t g_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
typedef struct { uint64_t key, ctr; } g_rng;
static g_rng g_rng_make(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
  g_rng r;
  r.key = g_mix(seed ^ g_mix(a * 0x100000001B3ull ^ g_mix(b + 0x632BE59BD9B4E019ull) ^ g_mix(c * 0xD6E8FEB86659FD93ull)));
  r.ctr = 0;
  return r;
}
static inline double g_uni(g_rng* r) { /* [0,1) with 53 random bits */
  uint64_t x = g_mix(r->key + (r->ctr++) * 0x9E3779B97F4A7C15ull);
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}
static inline double g_gauss(g_rng* r) { /* Box-Muller, one draw */
  double u1 = g_uni(r), u2 = g_uni(r);
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * G_PI * u2);
}

/* ----------------------------------------------------------- geometry */
static double g_row_x(int r) { return 85.0 + (double)r * 160.0 / 151.0; }
static int g_npads(int r) { return (int)floor(2.0 * g_row_x(r) * tan(10.0 * G_PI / 180.0) / 0.4); }
static double g_alpha(int s) { return ((double)(s % 18) * 20.0 + 10.0) * G_PI / 180.0; }

/* ------------------------------------------------------------- params */
typedef struct {
  uint64_t seed;
  int32_t n_coll;
  const double* t0;        /* [n_coll] collision times, us from TF start */
  const int32_t* ntracks;  /* [n_coll] primaries per collision           */
  double pt_mean;          /* GeV, exponential                           */
  double pt_min;           /* GeV, truncation                            */
  double eta_min, eta_max;
  int32_t sector_only;     /* -1: full TPC; else phi restricted to this sector and only its clusters kept */
  double zvtx_sigma;       /* cm */
  double sigma_y, sigma_z; /* cm */
  double noise_frac;       /* noise clusters = noise_frac * signal clusters */
  double bz;               /* T */
  double vdrift;           /* cm/us */
  double t_window;         /* us: clusters with time outside [0, t_window) are dropped */
  int32_t nthreads;
  int32_t angular_errors;  /* 1: smearing grows with the crossing angles (pad-length term) */
  double row_drop;         /* probability that a track's cluster on a row is lost */
} gen_params;

typedef struct {
  uint8_t sector, row;
  int32_t track;   /* global track id, -1 for noise */
  double y;        /* local y, cm */
  double zeta;     /* drift coordinate v_d * t, cm */
} g_cl;

typedef struct {
  g_cl* v;
  int64_t n, cap;
} g_buf;

static void g_push(g_buf* b, const g_cl* c) {
  if (b->n == b->cap) {
    b->cap = b->cap ? b->cap * 2 : 4096;
    b->v = (g_cl*)realloc(b->v, (size_t)b->cap * sizeof(g_cl));
  }
  b->v[b->n++] = *c;
}

typedef struct {
  double pt, eta, phi0, zv, t0;
  int32_t q, coll;
} g_truth;

typedef struct {
  gen_params P;
  int64_t ntrk_total;
  int64_t* trk_base;  /* [n_coll] first global track id */
  g_truth* truth;     /* [ntrk_total] */
  g_buf* bufs;        /* [n_coll] signal clusters per collision */
  int64_t n_signal, n_noise;
  g_cl* noise;        /* [n_noise] */
  int32_t npads[G_NROW];
  double rowx[G_NROW];
} g_state;

/* A particle from the beam axis: transverse circle through the origin, radius
 * R = pT / (0.00299792458 * |Bz|) cm.  For Bz > 0 a positive particle turns
 * clockwise seen from +z.  Clusters are recorded where the path first crosses
 * each pad-row plane of a sector, up to the turning point (half a turn), with
 * the crossing inside the pad plane and inside the drift volume. */
static void g_track(g_state* S, int32_t coll, int32_t it, int64_t gid, g_buf* out) {
  const gen_params* P = &S->P;
  g_rng R = g_rng_make(P->seed, 1, (uint64_t)coll, (uint64_t)it);
  double pt = P->pt_min - P->pt_mean * log(1.0 - g_uni(&R));
  double eta = P->eta_min + g_uni(&R) * (P->eta_max - P->eta_min);
  double phi0 = (P->sector_only >= 0) ? g_alpha(P->sector_only) + (2.0 * g_uni(&R) - 1.0) * (10.0 * G_PI / 180.0)
                                      : 2.0 * G_PI * g_uni(&R);
  int q = (g_uni(&R) < 0.5) ? -1 : 1;
  double zv = P->zvtx_sigma * g_gauss(&R);
  double t0 = P->t0[coll];
  double tanl = sinh(eta);
  g_truth* T = &S->truth[gid];
  T->pt = pt; T->eta = eta; T->phi0 = phi0; T->zv = zv; T->t0 = t0; T->q = q; T->coll = coll;

  int straight = (P->bz == 0.0);
  double Rc = straight ? 0.0 : pt / (0.00299792458 * fabs(P->bz));
  double h = straight ? 0.0 : ((P->bz > 0) ? -(double)q : (double)q); /* +1: counter-clockwise */
  double cx = h * Rc * -sin(phi0), cy = h * Rc * cos(phi0);

  /* Azimuth of the position swept out to the outer radius of the chamber:
   * from phi0 over h * asin(rho / 2R) (a quarter turn at most).  A sector
   * whose +-10 deg pad planes lie more than 2 deg outside that range gets no
   * cluster (2 deg at the innermost row is 3 cm, beyond any smearing), so it
   * is not visited. */
  double sweep = straight ? 0.0 : (2.0 * Rc <= G_RHO_MAX ? 0.5 * G_PI : asin(G_RHO_MAX / (2.0 * Rc)));
  double amid = phi0 + 0.5 * h * sweep;
  double awin = 0.5 * sweep + 12.0 * G_PI / 180.0;
  for (int j = 0; j < 18; ++j) {
    if (P->sector_only >= 0 && (P->sector_only % 18) != j) continue;
    if (fabs(remainder(g_alpha(j) - amid, 2.0 * G_PI)) > awin) continue;
    double a = g_alpha(j), ca = cos(a), sa = sin(a);
    double phil0 = phi0 - a;
    for (int r = 0; r < G_NROW; ++r) {
      double xr = S->rowx[r];
      double s_arc, yl, snp;
      if (straight) {
        double c = cos(phil0);
        if (c <= 0) continue;
        s_arc = xr / c;
        yl = s_arc * sin(phil0);
        snp = sin(phil0);
      } else {
        double xc = cx * ca + cy * sa, yc = -cx * sa + cy * ca;
        double v = (xr - xc) / (h * Rc);
        if (v < -1.0 || v > 1.0) continue;
        double cand[2] = {asin(v), G_PI - asin(v)};
        double best = -1.0, besty = 0.0, bests = 0.0;
        for (int k = 0; k < 2; ++k) {
          double sa_ = h * Rc * (cand[k] - phil0);
          double per = 2.0 * G_PI * Rc;
          sa_ = fmod(sa_, per);
          if (sa_ < 0) sa_ += per;
          if (sa_ <= 0.0 || sa_ > G_PI * Rc) continue;
          if (best < 0 || sa_ < best) { best = sa_; besty = yc - h * Rc * cos(cand[k]); bests = sin(cand[k]); }
        }
        if (best < 0) continue;
        s_arc = best; yl = besty; snp = bests;
      }
      double z = zv + s_arc * tanl;
      if (fabs(z) >= G_DRIFT_LEN) continue;
      int side_c = (z < 0);
      int sec = j + (side_c ? 18 : 0);
      if (P->sector_only >= 0 && sec != P->sector_only) continue;
      double sy = P->sigma_y, sz = P->sigma_z;
      if (P->angular_errors) {
        /* the pad-length term of the cluster errors: (L tan)^2 / 12 with L
         * the row pitch, tan(phi) of the crossing in the sector frame and
         * tan(lambda) of the track */
        const double l2 = (160.0 / 151.0) * (160.0 / 151.0) / 12.0;
        double s2 = snp * snp;
        sy = sqrt(sy * sy + l2 * (s2 < 1.0 ? s2 / (1.0 - s2) : 1e6));
        sz = sqrt(sz * sz + l2 * tanl * tanl);
      }
      double ys = yl + sy * g_gauss(&R);
      double zs = z + sz * g_gauss(&R);
      if (P->row_drop > 0.0 && g_uni(&R) < P->row_drop) continue;
      int np = S->npads[r];
      double pad = rint((ys + 0.2 * np) * 160.0);
      if (pad < 0 || pad > 64.0 * np - 1) continue;
      double zeta = P->vdrift * t0 + G_DRIFT_LEN + (side_c ? zs : -zs);
      double t = zeta / P->vdrift;
      if (!(t >= 0.0 && t < P->t_window)) continue;
      g_cl c;
      c.sector = (uint8_t)sec; c.row = (uint8_t)r; c.track = (int32_t)gid; c.y = ys; c.zeta = zeta;
      g_push(out, &c);
    }
  }
}

typedef struct { g_state* S; int tid, nth; } g_job;

static void* g_worker(void* arg) {
  g_job* J = (g_job*)arg;
  g_state* S = J->S;
  for (int32_t c = J->tid; c < S->P.n_coll; c += J->nth) {
    for (int32_t it = 0; it < S->P.ntracks[c]; ++it) g_track(S, c, it, S->trk_base[c] + it, &S->bufs[c]);
  }
  return NULL;
}

static void g_noise(g_state* S, int64_t i, g_cl* c) {
  const gen_params* P = &S->P;
  g_rng R = g_rng_make(P->seed, 2, (uint64_t)i, 0);
  int sec = (P->sector_only >= 0) ? P->sector_only : (int)(g_uni(&R) * G_NSEC);
  int r = (int)(g_uni(&R) * G_NROW);
  int np = S->npads[r];
  double pad = floor(g_uni(&R) * 64.0 * np);
  double t = g_uni(&R) * P->t_window;
  c->sector = (uint8_t)sec; c->row = (uint8_t)r; c->track = -1;
  c->y = pad / 160.0 - 0.2 * np;
  c->zeta = t * P->vdrift;
}

typedef struct { g_state* S; int64_t lo, hi; } g_njob;
static void* g_noise_worker(void* arg) {
  g_njob* J = (g_njob*)arg;
  for (int64_t i = J->lo; i < J->hi; ++i) g_noise(J->S, i, &J->S->noise[i]);
  return NULL;
}

/* Runs the simulation; returns an opaque handle, total cluster count in *n_out. */
void* o2gen_run(const gen_params* P, int64_t* n_out, int64_t* ntracks_out) {
  g_state* S = (g_state*)calloc(1, sizeof(g_state));
  S->P = *P;
  for (int r = 0; r < G_NROW; ++r) { S->rowx[r] = g_row_x(r); S->npads[r] = g_npads(r); }
  S->trk_base = (int64_t*)calloc((size_t)(P->n_coll > 0 ? P->n_coll : 1), sizeof(int64_t));
  int64_t tot = 0;
  for (int32_t c = 0; c < P->n_coll; ++c) { S->trk_base[c] = tot; tot += P->ntracks[c]; }
  S->ntrk_total = tot;
  S->truth = (g_truth*)calloc((size_t)(tot > 0 ? tot : 1), sizeof(g_truth));
  S->bufs = (g_buf*)calloc((size_t)(P->n_coll > 0 ? P->n_coll : 1), sizeof(g_buf));
  int nth = P->nthreads > 0 ? P->nthreads : 1;
  pthread_t* th = (pthread_t*)calloc((size_t)nth, sizeof(pthread_t));
  g_job* jobs = (g_job*)calloc((size_t)nth, sizeof(g_job));
  for (int t = 0; t < nth; ++t) { jobs[t].S = S; jobs[t].tid = t; jobs[t].nth = nth; pthread_create(&th[t], NULL, g_worker, &jobs[t]); }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  int64_t ns = 0;
  for (int32_t c = 0; c < P->n_coll; ++c) ns += S->bufs[c].n;
  S->n_signal = ns;
  S->n_noise = (int64_t)llround(P->noise_frac * (double)ns);
  S->noise = (g_cl*)calloc((size_t)(S->n_noise > 0 ? S->n_noise : 1), sizeof(g_cl));
  g_njob* nj = (g_njob*)calloc((size_t)nth, sizeof(g_njob));
  for (int t = 0; t < nth; ++t) {
    nj[t].S = S; nj[t].lo = S->n_noise * t / nth; nj[t].hi = S->n_noise * (t + 1) / nth;
    pthread_create(&th[t], NULL, g_noise_worker, &nj[t]);
  }
  for (int t = 0; t < nth; ++t) pthread_join(th[t], NULL);
  free(nj); free(th); free(jobs);
  *n_out = ns + S->n_noise;
  *ntracks_out = tot;
  return S;
}

/* Writes the clusters, in generation order (collision, track, sector, row;
 * then noise), into caller buffers.  Any pointer may be NULL.
 *   sector,row  : uint8
 *   y, z        : float; y local cm, z = apparent z in cm assuming the collision
 *                 happened at t = 0: side * (250 - v_d * t)  (side +1 A, -1 C)
 *   time        : float, us
 *   packed      : 12-byte records {u32 time64; u16 pad64; u16 charge; u8 row;
 *                 u8 sector; u16 spare}, time64 = rint(t * 320) (1/64 of a
 *                 200 ns time bin), pad64 = rint((y + 0.2 nPads) * 160) (1/64 pad)
 *   truth_track : int32 global track id or -1 (noise) */
void o2gen_copy(void* h, uint8_t* sector, uint8_t* row, float* y, float* z, float* time, uint8_t* packed,
                int32_t* truth_track) {
  g_state* S = (g_state*)h;
  int64_t o = 0;
  uint64_t charge_ctr = 0;
  for (int64_t c = 0; c <= S->P.n_coll; ++c) {
    const g_cl* v;
    int64_t n;
    if (c < S->P.n_coll) { v = S->bufs[c].v; n = S->bufs[c].n; }
    else { v = S->noise; n = S->n_noise; }
    for (int64_t i = 0; i < n; ++i, ++o) {
      const g_cl* cl = &v[i];
      int side = cl->sector < 18 ? 1 : -1;
      double t = cl->zeta / S->P.vdrift;
      if (sector) sector[o] = cl->sector;
      if (row) row[o] = cl->row;
      if (y) y[o] = (float)cl->y;
      if (z) z[o] = (float)(side * (G_DRIFT_LEN - cl->zeta));
      if (time) time[o] = (float)t;
      if (truth_track) truth_track[o] = cl->track;
      if (packed) {
        uint8_t* p = packed + 12 * o;
        uint32_t t64 = (uint32_t)rint(t * 320.0);
        uint16_t pad = (uint16_t)rint((cl->y + 0.2 * S->npads[cl->row]) * 160.0);
        uint16_t ch = (uint16_t)(g_mix(S->P.seed ^ (charge_ctr++)) & 0x3FF);
        uint16_t spare = 0;
        memcpy(p, &t64, 4); memcpy(p + 4, &pad, 2); memcpy(p + 6, &ch, 2);
        p[8] = cl->row; p[9] = cl->sector; memcpy(p + 10, &spare, 2);
      }
    }
  }
}

/* Per-track truth: pt, eta, phi0 (momentum azimuth at the vertex, global),
 * zv, t0 as doubles [ntracks][5]; charge and collision as int32. */
void o2gen_truth(void* h, double* dbl5, int32_t* q, int32_t* coll) {
  g_state* S = (g_state*)h;
  for (int64_t i = 0; i < S->ntrk_total; ++i) {
    const g_truth* T = &S->truth[i];
    if (dbl5) { dbl5[5 * i] = T->pt; dbl5[5 * i + 1] = T->eta; dbl5[5 * i + 2] = T->phi0; dbl5[5 * i + 3] = T->zv; dbl5[5 * i + 4] = T->t0; }
    if (q) q[i] = T->q;
    if (coll) coll[i] = T->coll;
  }
}

void o2gen_free(void* h) {
  g_state* S = (g_state*)h;
  if (!S) return;
  for (int32_t c = 0; c < S->P.n_coll; ++c) free(S->bufs[c].v);
  free(S->bufs); free(S->noise); free(S->truth); free(S->trk_base); free(S);
}
