/*
 * o2tpc_oracle.h - interface of the FP64 single-threaded CPU oracle tracker.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this; only the tests, the package entry's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 */
#ifndef O2TPC_ORACLE_H
#define O2TPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n;               /* clusters */
  int32_t format;          /* 0: float (sector,row,y,z); 1: fixed 12-byte records */
  const uint8_t* sector;   /* float format */
  const uint8_t* row;      /* float format */
  const float* y;          /* cm, local */
  const float* z;          /* cm, apparent z for a collision at t = 0 (NULL: use time) */
  const float* time;       /* us, drift time (float format without z) */
  const uint8_t* packed;   /* fixed format, n * 12 bytes */
  double bz;               /* T */
  double vdrift;           /* cm/us */
  uint64_t sector_mask;    /* bit s set: sector s is tracked (0 = all) */
  int32_t reverse_tracklet_order; /* 1: build tracklets in reverse order (selection order-independence test) */
  const double* coll_time; /* interaction times of the TF, us, ascending (may be NULL) */
  int64_t n_coll;
  int32_t compress;        /* 1: also build the compressed TF ("ctf", o2tpc_ctf.c) */
  int32_t row_step2;       /* 1: NeighboursFinder also links across one missing pad row */
  int32_t angular_errors;  /* 1: cluster errors grow with the track's angles */
} oracle_input;

typedef struct oracle_result oracle_result;

/* Runs the whole tracker.  *status: 0 ok, -1 invalid input. */
oracle_result* oracle_run(const oracle_input* in, int32_t* status);
void oracle_free(oracle_result* r);
/* Named outputs (see o2tpc_oracle.c, oracle_get).  Returns the element count
 * (-1 if unknown name); *ptr points into the result (owned by it);
 * *type: 0 int32, 1 int64, 2 double, 3 uint8. */
int64_t oracle_get(oracle_result* r, const char* name, const void** ptr, int32_t* type);

/* Building blocks, exposed so that the tests can pin them one by one. */
int32_t oracle_propagate(double* x, double* p5, double* c15, double x2, double bz);
int32_t oracle_update(double* p5, double* c15, double ym, double zm, double* chi2);
int32_t oracle_rotate(double* x, double* p5, double* c15, double dalpha);
/* Fits measurements (x_i, y_i, zeta_i) in the order given: the first point
 * seeds y and zeta, (sin phi, t, q/pT) come from p5; the initial covariance is
 * c15 if c15[0] > 0, else the tracker's initial diagonal.  Returns the state
 * and covariance at the last point in p5, c15. */
/* Compressed TF (o2tpc_ctf.c): encoder over plain arrays (per input cluster
 * sector, row, y, zeta in integer units; tracks as offsets + input indices;
 * q/pT per track; the sorted-hit order), decoder back to the cluster
 * sequence, and the entropy coder alone.  Buffers returned through out
 * pointers are malloc'd; the caller frees them.  Decoders return -1 on a
 * malformed input. */
int64_t oracle_ctf_encode(int64_t n_clusters, const int32_t* sector, const int32_t* row, const int32_t* y,
                          const int32_t* z, int64_t n_tracks, const int64_t* trk_off, const int32_t* trk_cl,
                          const double* trk_qpt, const int32_t* sorted_orig, int64_t n_sorted, uint8_t** out);
int64_t oracle_ctf_decode(const uint8_t* blob, int64_t bytes, int32_t** sector, int32_t** row, int32_t** y,
                          int32_t** z, int64_t* n_tracks, int64_t** trk_len);
void oracle_ctf_normalize(const uint64_t* count, uint16_t* freq);
int64_t oracle_rans_encode(const uint8_t* sym, int64_t n, uint8_t** out);
int64_t oracle_rans_decode(const uint8_t* blob, int64_t bytes, uint8_t** out);
void oracle_buffer_free(void* p);
/* Clusterizer (o2tpc_clu.c): digits sorted by (sector, row, time, pad) to
 * 12-byte cluster records; returns the cluster count, -1 on an unsorted or
 * out-of-range input. */
int64_t oracle_clusterize(int64_t n, const uint8_t* sector, const uint8_t* row, const uint8_t* pad,
                          const uint32_t* time, const uint16_t* adc, uint8_t** out);

/* Signed transverse arc length from (x0, y0) with sin(phi) = snp and
 * curvature k = dphi/ds to the closest approach to the origin. */
double oracle_dca_arc(double x0, double y0, double snp, double k);
int32_t oracle_fit_points(int32_t n, const double* x, const double* y, const double* z, double bz,
                          double* p5_inout, double* c15_out);

#ifdef __cplusplus
}
#endif
#endif
