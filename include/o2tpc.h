/*
 * o2tpc.h - C-ABI of the GB300 (sm_103a) TPC Time-Frame tracker.
 *
 * What the library computes.  TPC track reconstruction over one continuous-
 * readout Time Frame (TF): the paper's dominant synchronous workload
 * (Sec. 2.1), run on whole TFs of 128 LHC orbits, the processing unit of
 * Run 3 (Sec. 2), with tracks found before collisions are known, since the
 * drift time gives no a priori z (Sec. 2, Sec. 2.3).  Clusters go in (sector,
 * pad row, y, z or drift time); tracks come out as lists of cluster indices
 * plus helix parameters and covariance.  The steps, each a CUDA kernel:
 * grid binning and per-row sort, NeighboursFinder, NeighboursCleaner,
 * StartHitsFinder, TrackletConstructor (FP32 Kalman filter), TrackletSelector,
 * sector-to-sector merger and final refit (FP32, with an FP64 covariance
 * fallback that is counted).
 *
 * Execution model.  One context drives one GPU from one host thread, as the
 * paper's GPU code does (Sec. 3.1.1: one CPU core per GPU).  o2tpc_submit_tf
 * queues a TF and returns at once; a worker thread of the context admits
 * queued TFs by their device-memory footprint, runs the admitted ones as one
 * batch (one launch per step over all TFs in the batch) and copies the
 * results back; o2tpc_poll waits for one TF.  TFs whose footprint can never
 * fit are refused with O2TPC_ETOOBIG (the paper processes such TFs on the
 * CPU, Sec. 3.1.3); a full queue answers O2TPC_EAGAIN (back pressure,
 * Sec. 3.3).  Each TF's result is the same whether it ran alone or in a batch.
 *
 * Units and conventions.
 *   sector s: 0-17 side A (z > 0), 18-35 side C; sector s is centred at
 *     azimuth ((s mod 18) * 20 + 10) degrees; local x along the sector axis.
 *   pad row r: 0-151, plane at local x_r = 85 + r * 160/151 cm.
 *   y: local y in cm (pad direction).
 *   z (float input): apparent z in cm for a collision at t = 0,
 *     i.e. side * (250 - v_drift * t), side = +1 (A) / -1 (C).
 *   drift coordinate zeta = v_drift * t (cm); internally in units of 1/64 of
 *     a 200 ns time bin (3.125 ns).
 *   Output parameters, in the frame of the innermost cluster's sector at
 *   x = that cluster's pad-row x:
 *     par[0] y (cm)
 *     par[1] zeta - zeta_ref (cm), zeta_ref = the innermost cluster's drift
 *            coordinate (reported in time units of 1/64 bin in zeta_ref[])
 *     par[2] sin(phi) (local)
 *     par[3] tan(lambda) (dz/ds in the transverse path length)
 *     par[4] q/pT (1/GeV)
 *   cov: lower triangle of the 5x5 covariance, order
 *     (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1) (3,2) (3,3)
 *     (4,0) (4,1) (4,2) (4,3) (4,4).
 *
 * Errors.  Functions return O2TPC_OK (0), O2TPC_PENDING (1) or a negative
 * o2tpc_status.  No function aborts the process; a CUDA failure is reported
 * as O2TPC_ECUDA and leaves the context unusable (destroy it).
 */
#ifndef O2TPC_H
#define O2TPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct o2tpc_ctx o2tpc_ctx; /* opaque; owned by the library */

typedef enum {
  O2TPC_OK = 0,
  O2TPC_PENDING = 1,   /* poll: the TF is not done within the timeout          */
  O2TPC_EINVAL = -1,   /* bad argument, or a cluster with sector >= 36, row >= 152,
                          non-finite y/z or a drift coordinate out of range   */
  O2TPC_ENOMEM = -2,   /* a device or host allocation failed                   */
  O2TPC_EAGAIN = -3,   /* queue full: retry after polling/releasing             */
  O2TPC_ETOOBIG = -4,  /* the TF's footprint exceeds the memory budget          */
  O2TPC_ECUDA = -5,    /* a CUDA call failed                                    */
  O2TPC_ETIMEOUT = -6, /* a bounded device wait ran out                         */
  O2TPC_ENOTFOUND = -7 /* unknown ticket                                        */
} o2tpc_status;

enum { O2TPC_FMT_FLOAT = 0, O2TPC_FMT_FIXED = 1 };
enum { O2TPC_LOC_HOST = 0, O2TPC_LOC_DEVICE = 1 };

/* o2tpc_config.flags */
enum {
  O2TPC_FLAG_KEEP_STAGES = 1u << 0, /* keep per-step device arrays until release,
                                       readable with o2tpc_get_stage          */
  O2TPC_FLAG_NO_BATCHING = 1u << 1, /* run every TF alone (one TF per batch)  */
  O2TPC_FLAG_FORCE_FP64 = 1u << 2,  /* take the FP64 covariance path in the final
                                       refit for every track (testing aid)     */
  O2TPC_FLAG_AUTOTUNE = 1u << 3,    /* on the first batch of >= 2^20 clusters,
                                       time the launch shapes of the tunable
                                       steps on that batch and keep the fastest
                                       (see o2tpc_get_tuning)                  */
  O2TPC_FLAG_GRAPH_TIGHT = 1u << 4, /* captured path with token capacities (16
                                       tracklets, sector tracks, pairs): batches
                                       overflow and rerun on the regular path
                                       (testing aid)                           */
  O2TPC_FLAG_COOP_SEARCH = 1u << 6, /* following passes of the tracklet
                                       constructor: the candidate hits of all
                                       lanes' row windows scanned together by
                                       the warp, instead of each lane scanning
                                       its own (identical results)             */
  O2TPC_FLAG_ROW_STEP2 = 1u << 7,  /* NeighboursFinder: a hit without an accepted
                                       pair on the adjacent rows may link across
                                       one missing pad row (rows r + a, r - b,
                                       (a, b) in {(2,1), (1,2), (2,2)}, residual
                                       (a + b) h - b u - a d, its chi2 scaled by
                                       6 / ((a + b)^2 + a^2 + b^2)).  A reading:
                                       the paper only asks for robustness at
                                       five-fold occupancy (Sec. 2.3)          */
  O2TPC_FLAG_ANGULAR_ERRORS = 1u << 8, /* cluster errors grow with the track
                                       angles: variances + (L tan phi)^2 / 12 in
                                       y and (L tan lambda)^2 / 12 in zeta, L the
                                       pad length 160/151 cm, at the predicted
                                       state (a reading, as above)             */
  O2TPC_FLAG_COMPRESS = 1u << 5     /* also build each TF's compressed form
                                       (o2tpc_result.ctf; Sec. 2.2: clusters of
                                       tracks with pT < 0.1 GeV removed, a
                                       straight-line integer track model, rANS;
                                       format in csrc/k_ctf.cu).  Batches take
                                       the regular path; 48 more device bytes
                                       per cluster; a TF above 250 M clusters
                                       is refused with ETOOBIG                 */
};

typedef struct {
  int32_t device;          /* CUDA device ordinal                                     */
  uint64_t mem_budget;     /* device bytes the admitted TFs may use (0: 120 GB)       */
  int32_t max_inflight;    /* TFs queued or running at once (0: 64)                   */
  int32_t max_batch;       /* TFs per batch (0: 64); a batch also stops taking TFs
                              once it holds batch_full_clusters clusters or would
                              exceed mem_budget                                      */
  double bz_tesla;         /* solenoid field (0 allowed: straight lines)              */
  double vdrift_cm_us;     /* drift velocity (> 0)                                    */
  uint32_t flags;          /* O2TPC_FLAG_*                                            */
  /* Device memory: if dev_alloc is set, every device buffer comes from it
   * (e.g. a framework's caching allocator) and goes back through dev_free,
   * and host-resident inputs are copied in the batch's own stream.
   * Otherwise buffers come from a stream-ordered memory pool the context
   * owns (freed memory is kept for the next batch until o2tpc_destroy), and
   * host-resident inputs still waiting in the queue are uploaded ahead on a
   * second (copy) stream while earlier batches compute; these copies use up
   * to mem_budget / 8 device bytes beyond mem_budget.  dev_alloc must
   * return blocks aligned to 256 bytes, as cudaMalloc does; a block that
   * is not 16-byte aligned is handed back to dev_free and the call fails
   * with O2TPC_ENOMEM. */
  void* (*dev_alloc)(size_t bytes, void* user);
  void (*dev_free)(void* ptr, void* user);
  void* alloc_user;
  void* stream;            /* cudaStream_t to run on, or NULL for a library stream    */
  uint64_t batch_full_clusters; /* clusters that fill the GPU: a TF joins a batch
                              only if the batch stays within this many clusters (a
                              larger TF runs alone) (0: 2^25; UINT64_MAX: only
                              max_batch and mem_budget limit a batch)                 */
  /* Launch shapes (0: default, or the autotuner's choice with
   * O2TPC_FLAG_AUTOTUNE).  Results never depend on them. */
  int32_t nf_hits_per_block;     /* NeighboursFinder: hits (threads) per block of a
                                    pad row: 64, 128 (default) or 256             */
  int32_t sort_threads_per_row;  /* cell sort: threads per pad row: 128, 256
                                    (default) or 512                              */
  /* Captured path (0: off): batches of at most graph_max_tfs TFs (0: 64) and
   * graph_max_clusters clusters run as ONE CUDA graph launch - the whole
   * pipeline captured once and replayed, no host synchronisation inside -
   * from a device arena allocated at o2tpc_create (about 220 bytes per
   * cluster of graph_max_clusters, on top of mem_budget).  A batch whose
   * data exceed the arena's capacities (e.g. far more tracklets than usual)
   * is run again on the regular path; results are the same either way.
   * Not used with O2TPC_FLAG_KEEP_STAGES. */
  uint64_t graph_max_clusters;
  int32_t graph_max_tfs;
  int32_t nf_staged;             /* NeighboursFinder candidates staged in shared
                                    memory by TMA bulk copies (1) or read through
                                    L1 (0, default); the autotuner times both    */
  const char* tune_cache_path;   /* NULL, or a text file keeping the autotuner's
                                    choice per GPU model: read at o2tpc_create
                                    (a matching entry counts as tuned), written
                                    after tuning                                  */
  uint32_t debug_inject;         /* fault injection for tests (0: none).  Bit 0:
                                    the staged NeighboursFinder arms its slab
                                    barrier but issues no copy, and its bounded
                                    waits give up after 64 polls: every wait runs
                                    out with nothing in flight, the blocks read
                                    global memory instead (same links) and the
                                    batch reports o2tpc_stats.events bit 0.  Takes
                                    effect with nf_staged = 1, on the regular path */
} o2tpc_config;

/* Launch shapes in use and, once the autotuner has run, its timings (device
 * ms of each candidate on the batch it tuned on). */
typedef struct {
  int32_t tuned;                 /* 1 once the autotuner has chosen               */
  int32_t nf_hits_per_block;
  int32_t nf_staged;
  int32_t sort_threads_per_row;
  int32_t tuned_on_clusters;     /* size of the batch it tuned on                 */
  float nf_ms[6];                /* 64, 128, 256 hits per block; L1 then staged   */
  float sort_ms[3];              /* 128, 256, 512 threads per row                 */
} o2tpc_tuning;

typedef struct {
  uint64_t n;              /* clusters (may be 0)                                      */
  int32_t format;          /* O2TPC_FMT_FLOAT or O2TPC_FMT_FIXED                       */
  int32_t location;        /* O2TPC_LOC_HOST or O2TPC_LOC_DEVICE (pointers below)      */
  /* FLOAT: arrays of n */
  const uint8_t* sector;
  const uint8_t* row;
  const float* y;          /* cm                                                       */
  const float* z;          /* cm, apparent z (see above); may be NULL when time is set  */
  const float* time;       /* drift time in us (used when z is NULL): zeta units =
                              rintf(time * 320), as the fixed format's time64          */
  /* FIXED: n records of 12 bytes, little endian:
   *   u32 time64 (drift time in 1/64 of a 200 ns bin, < 2^30), u16 pad64
   *   (pad position in 1/64 pad, 0 at the sector's pad-plane edge), u16 charge,
   *   u8 row, u8 sector, u16 spare */
  const void* packed;
  uint64_t user_tag;       /* echoed in the result                                     */
  /* Interaction record (Sec. 2: tracks are assigned to collisions after
   * tracking): n_coll collision times of this TF in us from its start,
   * ascending and finite, in HOST memory whatever `location` says (copied at
   * the batch start; borrowed like the clusters).  May be NULL with n_coll 0:
   * every track's collision is then -1.  Unsorted or non-finite -> EINVAL. */
  const double* coll_time;
  uint64_t n_coll;
} o2tpc_tf;

typedef struct {
  uint64_t n_clusters;
  uint64_t n_tracklets;      /* start hits = tracklets built                          */
  uint64_t n_sector_tracks;
  uint64_t n_tracks;
  uint64_t n_fp64_fallback;  /* tracks whose final refit ran with FP64 covariance     */
  uint32_t batch_size;       /* TFs in the batch this TF ran in                       */
  float ms_queue;            /* submit -> batch start (host clock)                    */
  float ms_batch;            /* batch start -> results on the host (host clock)       */
  float ms_device;           /* device time of the batch (CUDA events)                */
  uint64_t n_launches;       /* kernels launched for the batch                        */
  /* device time of each step of the batch (CUDA events on the context's stream,
   * gaps for the host reading sizes included): 0 ingest + row statistics +
   * grid, 1 row/cell sort, 2 NeighboursFinder, 3 NeighboursCleaner +
   * StartHitsFinder, 4 TrackletConstructor, 5 TrackletSelector, 6 sector-track
   * fits, 7 merger, 8 final refit, 9 read-back of the result sizes,
   * 10 result download; 11 is host time (not device) spent preparing the
   * result copies (pinned blocks, offsets) inside step 10; 12 upload: from
   * the batch start to the start of step 0 (host-resident inputs copied in
   * the batch's own stream, descriptor tables); 13 time the batch waited for
   * inputs that were uploaded ahead on the context's copy stream; 14 and 15
   * the outward and the inward following passes inside step 4; 16 the
   * continuous-readout step (t0, membrane links, collision assignment) that
   * follows step 8; 17 the compressed-TF step (O2TPC_FLAG_COMPRESS) */
  float ms_stage[18];
  uint32_t captured;         /* 1: the batch ran as one CUDA graph launch (the
                                captured path: ms_stage holds only 10-13)     */
  uint32_t events;           /* bit0: a bounded device wait ran out in the batch
                                (the NeighboursFinder's staged copy; the step
                                then read global memory, results complete)  */
} o2tpc_stats;

/* Result of one TF; library-owned memory, valid until o2tpc_result_release. */
typedef struct {
  uint64_t n_tracks;
  const uint64_t* offsets;     /* [n_tracks + 1] into cluster_idx                     */
  const uint32_t* cluster_idx; /* indices into the submitted cluster order, innermost
                                  segment first, ascending pad row within a sector   */
  const float* x;              /* [n_tracks] local x of the reported state (cm)       */
  const float* alpha;          /* [n_tracks] sector frame angle (rad)                 */
  const float* par;            /* [n_tracks][5]                                       */
  const float* cov;            /* [n_tracks][15]                                      */
  const float* chi2;           /* [n_tracks]                                          */
  const int32_t* ndf;          /* [n_tracks] 2 * fitted clusters - 5                  */
  const uint8_t* sector;       /* [n_tracks] sector of the reported frame             */
  const uint8_t* flags;        /* [n_tracks] bit0 FP64 fallback, bit1 merged from
                                  several sectors, bit2 refit stopped at a sector
                                  boundary, bit3 linked across the central
                                  membrane (t0 from the crossing)                    */
  const uint32_t* zeta_ref;    /* [n_tracks] drift coordinate origin of par[1]        */
  /* Continuous readout (Sec. 2).  Every cluster has 0 <= |z| <= 250 cm, so
   * the drift coordinates of the track's two end clusters (the extremes of
   * a helix) bound the collision time: t0_lo <= t0 <= t0_hi.
   * A track linked across the central membrane (mate >= 0, flags bit3) gets
   * t0 from where its two halves meet; any other track from its closest
   * approach to the beam axis with z_vertex = 0 assumed (error including a
   * 5 cm beam spot), clamped into the bounds.  collision: index into the
   * TF's coll_time of the compatible time (within the bounds +- 0.3 us)
   * nearest to t0, -1 if none.                                              */
  const float* t0;             /* [n_tracks] us from the TF start                    */
  const float* t0_err;         /* [n_tracks] us                                      */
  const float* t0_lo;          /* [n_tracks] us                                      */
  const float* t0_hi;          /* [n_tracks] us                                      */
  const int32_t* mate;         /* [n_tracks] the other half across the membrane, -1 */
  const int32_t* collision;    /* [n_tracks] interaction index, -1                   */
  /* With O2TPC_FLAG_COMPRESS: the TF's compressed form (NULL / 0 otherwise).
   * Lossless for the kept clusters' integer coordinates (sector, row, y in
   * 1/160 cm, zeta in 1/64 time bin); clusters of tracks with pT < 0.1 GeV
   * are left out.                                                           */
  const uint8_t* ctf;
  uint64_t ctf_bytes;
  o2tpc_stats stats;
  uint64_t user_tag;
  int32_t status;              /* O2TPC_OK or the error of this TF                    */
} o2tpc_result;

/* Raw ADC digits for the clusterizer (Sec. 2.2: raw ADC values are turned
 * into hits before tracking).  DEVICE arrays of n entries, zero-suppressed,
 * sorted strictly ascending by (sector, row, time, pad); sector < 36,
 * row < 152, time < 2^24 (200 ns bins). */
typedef struct {
  uint64_t n;
  const uint8_t* sector;
  const uint8_t* row;
  const uint8_t* pad;      /* pad in its row, 0 at the pad-plane edge          */
  const uint32_t* time;    /* time bin                                          */
  const uint16_t* adc;     /* ADC counts                                        */
} o2tpc_digits;

/* Clusterizer: one 12-byte cluster record (the O2TPC_FMT_FIXED layout: u32
 * time64, u16 pad64, u16 charge, u8 row, u8 sector, u16 0) per charge peak,
 * in the order of the peaks, written to the DEVICE buffer records (4-byte
 * aligned, room for cap records; its output can be submitted as a TF).  A
 * peak is a digit with ADC >= 3 larger than each of its up to eight pad/time
 * neighbours of the same row that come before it in the sorted order and not
 * smaller than each that comes after it; its record carries the charge sum
 * and the centre of gravity of the 3 x 3 cells around it, rounded half up in
 * 1/64 pad and 1/64 time bin.  Runs on `stream` (a cudaStream_t, NULL for the
 * default stream) with scratch from the stream-ordered allocator and returns
 * when the records are written.  *n_clusters: the number of peaks (also when
 * it exceeds cap).  Returns O2TPC_OK, O2TPC_EINVAL (null pointers, misaligned
 * records, unsorted or out-of-range digits), O2TPC_ETOOBIG (n >= 2^31, or more
 * peaks than cap: nothing written), O2TPC_ENOMEM, O2TPC_ECUDA. */
int o2tpc_clusterize(const o2tpc_digits* digits, void* records, uint64_t cap, uint64_t* n_clusters, void* stream);

/* A compressed TF decoded on the host (o2tpc_ctf_decode): the cluster
 * sequence of the format - the kept tracks' clusters first (track by track,
 * n_tracks tracks of track_len[i] clusters), then the clusters on no track -
 * as integer coordinates: sector, row, y in 1/160 cm, zeta in 1/64 time bin
 * (the fixed format's pad64 = y + 32 nPads(row), time64 = zeta).  Arrays are
 * owned by the library until o2tpc_ctf_free. */
typedef struct {
  uint64_t n;
  uint64_t n_tracks;
  const int32_t* sector;
  const int32_t* row;
  const int32_t* y;
  const int32_t* zeta;
  const uint32_t* track_len;
} o2tpc_ctf_clusters;

/* Decodes a compressed TF (o2tpc_result.ctf) on the host; no device work, no
 * context needed.  Returns O2TPC_OK, O2TPC_EINVAL (not a compressed TF, or
 * damaged: every chunk's coder must end in its initial state with its bytes
 * used up, and the payloads must end the blob), O2TPC_ENOMEM.  *out is
 * zeroed on error. */
int o2tpc_ctf_decode(const uint8_t* blob, uint64_t bytes, o2tpc_ctf_clusters* out);
void o2tpc_ctf_free(o2tpc_ctf_clusters* clusters);
/* The decoded clusters as O2TPC_FMT_FIXED records (12 bytes each, host
 * buffer of 12 n bytes; charge 0): pad64 = y + 32 nPads(row), nPads(row) =
 * floor(2 x_row tan(10 deg) / 0.4 cm), time64 = zeta; a decoded TF can be
 * submitted again.  Returns O2TPC_OK or O2TPC_EINVAL (a value out of the
 * record's range). */
int o2tpc_ctf_records(const o2tpc_ctf_clusters* clusters, void* records);

/* Creates a context on cfg->device (cfg may be NULL: all defaults).
 * *out is set on success.  Returns O2TPC_EINVAL, O2TPC_ECUDA or O2TPC_ENOMEM. */
int o2tpc_create(const o2tpc_config* cfg, o2tpc_ctx** out);

/* Queues one TF.  The input is borrowed, not copied: host input (pinned
 * memory gives the fastest upload) and device input alike must stay valid and
 * unchanged until o2tpc_poll has returned the TF's result.  *ticket
 * identifies the TF.
 * Returns O2TPC_OK, O2TPC_EINVAL, O2TPC_EAGAIN (queue full), O2TPC_ETOOBIG,
 * O2TPC_ENOMEM.  Invalid cluster content is detected on the device and
 * reported by o2tpc_poll as the TF's status O2TPC_EINVAL. */
int o2tpc_submit_tf(o2tpc_ctx* ctx, const o2tpc_tf* tf, uint64_t* ticket);

/* Queues n TFs at once (tfs[0..n-1], tickets[0..n-1] set on success): the
 * worker sees all of them together, so they go into one batch as far as
 * max_batch, batch_full_clusters and mem_budget allow (e.g. the chunks of one
 * Time Frame processed in a single launch sequence).  All or nothing: on any
 * error no TF is queued.  Same returns and borrowing rules as
 * o2tpc_submit_tf; O2TPC_EAGAIN if the n TFs do not fit in max_inflight. */
int o2tpc_submit_many(o2tpc_ctx* ctx, const o2tpc_tf* tfs, uint32_t n, uint64_t* tickets);

/* Waits up to timeout_ms (< 0: forever, 0: just test) for a TF.  On
 * O2TPC_OK, *out is the result (its own status may still be an error).
 * Returns O2TPC_PENDING on timeout, O2TPC_ENOTFOUND for an unknown ticket. */
int o2tpc_poll(o2tpc_ctx* ctx, uint64_t ticket, int32_t timeout_ms, const o2tpc_result** out);

/* Frees a polled result (and the TF's kept stages); the ticket is retired. */
void o2tpc_result_release(o2tpc_ctx* ctx, const o2tpc_result* res);

/* Waits for all queued work, frees everything.  Returns O2TPC_OK or the first
 * CUDA error seen. */
int o2tpc_destroy(o2tpc_ctx* ctx);

/* Human-readable text of a status code (static storage). */
const char* o2tpc_strerror(int32_t status);

/* Intermediate arrays of one polled TF, kept when the context was created
 * with O2TPC_FLAG_KEEP_STAGES (for testing and inspection).  Copies the named
 * array to host memory dst (capacity bytes); *needed receives its size in
 * bytes.  Indices are local to the TF (hit indices count from its first
 * sorted hit).  Returns O2TPC_OK, O2TPC_EINVAL (unknown name or dst too
 * small; *needed still set), O2TPC_ENOTFOUND.  Names:
 *   "sorted_orig"  int32[n]  input index of each sorted hit
 *   "sorted_yz"    int32[n][2] y and zeta in integer units, sorted order
 *   "row_grid"     int32[5472][8] start, count, cellBase, ny, nz, cz, zmin, 0
 *   "cell_start"   int32[cells + 1]
 *   "up_raw", "dn_raw", "up", "dn"  int32[n]
 *   "starts"       int32[n_tracklets]
 *   "tl_nhits"     int32[n_tracklets]  (0 if dropped)
 *   "tl_hits"      int32[n_tracklets][152] hit slots, ascending rows, -1 padded
 *   "tl_state"     float[n_tracklets][21]  x, par[5], cov[15] (zeta rel. start hit)
 *   "st_tracklet"  int32[n_sector_tracks]
 *   "st_off"       int32[n_sector_tracks + 1]
 *   "st_hits"      int32[...] sorted hit indices of the sector tracks
 *   "st_in", "st_out" float[n_sector_tracks][21]
 *   "st_next", "st_prev" int32[n_sector_tracks] merge links (-1 none)
 */
int o2tpc_get_stage(o2tpc_ctx* ctx, uint64_t ticket, const char* name, void* dst, uint64_t capacity,
                    uint64_t* needed);

/* Current launch shapes and autotuner timings (see o2tpc_tuning).  The paper
 * has no counterpart: its block shapes are fixed per GPU model.  Returns
 * O2TPC_OK or O2TPC_EINVAL. */
int o2tpc_get_tuning(o2tpc_ctx* ctx, o2tpc_tuning* out);

/* Allocation-free grid binning and stable sort of one TF.
 *
 * The paper has no counterpart of this entry point.  It is for callers that
 * cannot allocate device memory while they run (a host framework that owns
 * every device buffer, a fixed memory plan, code that must not synchronise
 * the device through cudaMalloc or grow its footprint after start-up): the
 * step's scratch memory is a set of file-scope static device arrays of fixed
 * size (about 6 MB, held by every GPU that loads the library until the
 * process exits), so this call allocates nothing, neither directly nor
 * through any allocating library routine.
 *
 * It computes, for one TF, what o2tpc_get_stage reports after a full run as
 * "sorted_orig", "sorted_yz", "row_grid" and "cell_start".
 *   tf           n <= O2TPC_STATIC_MAX_CLUSTERS (else O2TPC_ETOOBIG), location
 *                O2TPC_LOC_DEVICE; its buffers are read, not modified.
 *   vdrift_cm_us drift velocity (> 0) of the float-input quantisation.
 *   sorted_orig  device int32[n]: input index of each sorted hit.
 *   sorted_yz    device int32[n][2]: y and zeta in integer units, sorted.
 *   row_grid     device int32[5472][8]: start, count, cellBase, ny, nz, cz,
 *                zmin, 0 per (sector, row).
 *   cell_start   device int32[cell_capacity] with cell_capacity >=
 *                n / 4 + 46 * 5472 + 2 (else O2TPC_EINVAL): the first sorted
 *                hit of every cell, plus the total at index cells.
 *   stream       cudaStream_t to run on (NULL: the default stream).
 * The call returns when the work is done: O2TPC_OK, O2TPC_EINVAL (bad
 * arguments or invalid cluster content), O2TPC_ETOOBIG, O2TPC_ECUDA.
 * The static arrays' device addresses are looked up during the first call on
 * each device (with that device current), so make that first call before any
 * stream capture.  With CUDA's lazy module loading (the default) that first
 * call may also load the library's device code and reserve the ~6 MB of
 * static storage at that moment: a caller with a fixed memory plan makes one
 * call with n = 0 at start-up (or runs with CUDA_MODULE_LOADING=EAGER).  The
 * looked-up addresses are kept for the life of the process and are not valid
 * after a cudaDeviceReset.  Every call copies its small descriptors (the TF,
 * its tiles, the geometry) from host memory and waits for its stream to
 * finish before it returns.  Every call shares the arrays and leaves its
 * contents in them: calls that overlap on the GPU race and must be
 * serialised. */
#define O2TPC_STATIC_MAX_CLUSTERS 262144
int o2tpc_sort_tf_static(const o2tpc_tf* tf, double vdrift_cm_us, int32_t* sorted_orig, int32_t* sorted_yz,
                         int32_t* row_grid, int32_t* cell_start, uint64_t cell_capacity, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* O2TPC_H */
