// o2tpc_capi.cu - host runtime behind include/o2tpc.h.
//
// One context owns one CUDA stream and one worker thread (the paper drives
// each GPU from one CPU core, Sec. 3.1.1).  Submitted Time Frames wait in a
// FIFO; the worker admits as many as fit the memory budget and the batch
// limits and runs them as one batch: every step is one launch over all TFs
// of the batch (rows are indexed tf * 5472 + sector * 152 + row, so no step
// mixes TFs and each TF's result does not depend on its batch mates).  Four
// host synchronisations per batch read the data-dependent sizes (start hits,
// sector tracks, merge pairs, tracks) that the following buffers need.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "o2tpc.h"
#include "o2tpc_graph.cuh"
#include "o2tpc_kernels.cuh"

using namespace o2tpc;

thread_local long long o2tpc::g_launch_count = 0;

void o2tpc::fill_geom(GeomConst& g, double bz, double vd) {
  const double pi = 3.14159265358979323846;
  std::memset(&g, 0, sizeof(g));
  for (int r = 0; r < kNRow; ++r) {
    double x = 85.0 + (double)r * 160.0 / 151.0;
    g.rowx[r] = (float)x;
    g.rowx_d[r] = x;
    g.npads[r] = (int)std::floor(2.0 * x * std::tan(10.0 * pi / 180.0) / 0.4);
  }
  g.pitch_d = 160.0 / 151.0;
  g.pitch = (float)g.pitch_d;
  for (int s = 0; s < 18; ++s) g.sec_alpha[s] = (float)((s * 20.0 + 10.0) * pi / 180.0);
  g.tan10 = (float)std::tan(10.0 * pi / 180.0);
  g.rot_cos = (float)std::cos(20.0 * pi / 180.0);
  g.rot_sin = (float)std::sin(20.0 * pi / 180.0);
  g.rot_cos_d = std::cos(20.0 * pi / 180.0);
  g.rot_sin_d = std::sin(20.0 * pi / 180.0);
  g.bzc_d = -0.00299792458 * bz;
  g.bzc = (float)g.bzc_d;
  g.zunit_d = 0.003125 * vd;
  g.zunit = (float)g.zunit_d;
  g.vd_d = vd;
  g.kz = (float)(1.0 / (0.003125 * vd));
}

namespace {

constexpr int kTileMin = 65536;           // clusters per ingest tile, at least
constexpr int kTilesPerTFMax = 4096;
constexpr uint64_t kMaxBatchHits = 2000000000ull;
// With the compressed TF: the blob offsets are 32-bit, and a coded cluster
// takes at most about 8.2 bytes (ten byte planes at <= 8 bits plus table
// rounding), so batches stay below 250 M clusters.
constexpr uint64_t kMaxCompressHits = 250000000ull;
// Default for o2tpc_config::batch_full_clusters: this many clusters fill the
// GPU; larger batches would only add latency (the TFs left out wait, uploaded
// ahead).
constexpr uint64_t kBatchFullHits = 1ull << 25;

struct CudaError {
  cudaError_t e;
  int line;
};
#define CK(x)                                             \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) throw CudaError{e_, __LINE__}; \
  } while (0)
// checks the last launch
#define CKL() CK(cudaGetLastError())

struct AllocError {};

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ----------------------------------------------------------- allocations
struct Ctx;

struct DevBlock {
  void* p = nullptr;
  size_t bytes = 0;
};

// All device buffers of one batch; freed when the last of its TFs is released
// (or at once when stages are not kept).
struct BatchMem {
  Ctx* ctx = nullptr;
  std::vector<DevBlock> blocks;
  int refs = 0;
  // stage views (valid while kept)
  int nTF = 0, nRows = 0, N = 0, nTl = 0, nSt = 0, nCells = 0;
  std::vector<int> tfHitBase, tfHitEnd, tfInBase, tfTlBegin, tfStBegin, tfCellBase, tfCellEnd;
  RowGrid* grid = nullptr;
  int *cellStart = nullptr, *sorig = nullptr, *upRaw = nullptr, *dnRaw = nullptr, *up = nullptr, *dn = nullptr;
  int2* syz = nullptr;
  int* starts = nullptr;
  TrackletBufs tb{};
  SectorTrackBufs sb{};
  MergeBufs mb{};
  ~BatchMem();
  void* alloc(size_t bytes);
};

struct Job {
  uint64_t ticket = 0;
  o2tpc_tf tf{};
  uint64_t footprint = 0;
  double t_submit = 0, t_start = 0, t_end = 0;
  bool done = false;
  int status = O2TPC_OK;
  // result storage: one pinned host block from the context's pool
  o2tpc_result res{};
  void* host = nullptr;
  size_t hostBytes = 0;
  uint64_t emptyOffset = 0;
  std::shared_ptr<BatchMem> mem;  // kept stages
  int tfIndex = 0;
  // upload ahead (host-resident input copied on the context's copy stream
  // while earlier batches compute): 0 not started, 1 being issued, 2 issued,
  // 3 left to the batch's own stream, 4 copy owned by the batch's memory
  int upState = 0;
  void* dIn = nullptr;
  uint64_t dInBytes = 0;
  cudaEvent_t upEv = nullptr;
};

// Device bytes of a host-resident TF's input copy.
uint64_t input_bytes(const o2tpc_tf& t) {
  return t.format == O2TPC_FMT_FIXED ? 12ull * t.n : 10ull * t.n + 64;
}

// A batch whose results are being copied to the host on the download stream.
struct Pending {
  std::vector<std::shared_ptr<Job>> jobs;
  std::shared_ptr<BatchMem> out;  // device result arrays, freed once copied
  cudaEvent_t dl0 = nullptr, dl1 = nullptr;
  cudaEvent_t trS = nullptr, trE = nullptr;  // timeline: batch start and compute end on the stream
  double hS = 0.0, hD = 0.0;                 // host clock: batch start, downloads issued
  float stageMs[18] = {};
  double hostPrepMs = 0;
  bool captured = false;
  ~Pending() {
    if (dl0) cudaEventDestroy(dl0);
    if (dl1) cudaEventDestroy(dl1);
    if (trS) cudaEventDestroy(trS);
    if (trE) cudaEventDestroy(trE);
  }
};

struct Ctx {
  o2tpc_config cfg{};
  cudaStream_t stream = nullptr;
  bool ownStream = false;
  GeomConst* dGeom = nullptr;
  Counts* dCounts = nullptr;  // sizes of the running regular-path batch
  GeomConst hGeom{};
  std::thread worker;
  std::mutex mu;
  std::condition_variable cvWork, cvDone;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t nextTicket = 1;
  int inflight = 0;
  bool stop = false;
  int fatal = O2TPC_OK;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evWait = nullptr;
  cudaEvent_t evs[12] = {};
  cudaEvent_t evTl[4] = {};  // ends of the four tracklet passes
  cudaEvent_t evCtf[2] = {};  // the compression step
  o2tpc_tuning tune{};       // launch shapes in use (autotuner results)
  // captured path: arena and two graphs, identical but for the set of result
  // arrays they write (replays alternate between them, so a replay never
  // waits for the previous replay's results to download), and per set the
  // event after the result copies of its last replay
  std::unique_ptr<GraphArena> graph;
  void* graphMem = nullptr;
  cudaGraphExec_t graphExec[2] = {nullptr, nullptr};
  long long graphKernels = 0;
  int graphNf = 0, graphSort = 0;
  cudaEvent_t graphDl[2] = {nullptr, nullptr};
  bool graphDlRecorded[2] = {false, false};
  int graphSlot = 0;  // the set the next replay writes
  // copy stream, its thread and the bytes uploaded ahead of their batch
  cudaStream_t upStream = nullptr;
  std::thread uploader;
  std::condition_variable cvUp;
  uint64_t upAheadBytes = 0, upAheadLimit = 0;
  // the library's own stream-ordered pool (no user allocator)
  cudaMemPool_t pool = nullptr;
  // result download: a third stream and the thread that completes batches
  // once their copies have landed (the worker starts the next batch meanwhile)
  cudaStream_t dlStream = nullptr;
  std::thread finisher;
  std::condition_variable cvFin;
  std::deque<std::shared_ptr<Pending>> finQueue;
  bool finStop = false;
  bool traceCopies = false;  // O2TPC_TRACE_COPIES=1: time every result copy (stderr);
  int traceMode = 0;         // =2: per-batch device timeline (stderr)
  cudaEvent_t evRef = nullptr;  // timeline origin
  double hostRef = 0.0;         // host clock when evRef was recorded
  // pinned staging for descriptors and results
  void* hStage = nullptr;
  size_t hStageBytes = 0;

  void* dev_alloc(size_t bytes) { return dev_alloc_on(bytes, stream); }
  void* dev_alloc_on(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (cfg.dev_alloc) {
      p = cfg.dev_alloc(bytes, cfg.alloc_user);
      if (p && (reinterpret_cast<uintptr_t>(p) & 15)) {  // vector and bulk copies need 16 B
        if (cfg.dev_free) cfg.dev_free(p, cfg.alloc_user);
        p = nullptr;
      }
    } else {
      if (cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
      }
    }
    if (!p) throw AllocError{};
    return p;
  }
  void dev_free(void* p) {
    if (!p) return;
    if (cfg.dev_free) cfg.dev_free(p, cfg.alloc_user);
    else cudaFreeAsync(p, stream);
  }
  // Pool of pinned host blocks for results (sizes rounded to 1 MiB).
  std::mutex poolMu;
  std::multimap<size_t, void*> pinnedFree;
  void* pinned_get(size_t bytes, size_t* got) {
    size_t want = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    {
      std::lock_guard<std::mutex> lk(poolMu);
      auto it = pinnedFree.lower_bound(want);
      if (it != pinnedFree.end() && it->first <= 2 * want) {
        void* p = it->second;
        *got = it->first;
        pinnedFree.erase(it);
        return p;
      }
    }
    void* p = nullptr;
    CK(cudaMallocHost(&p, want));
    *got = want;
    return p;
  }
  void pinned_put(void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(poolMu);
    pinnedFree.emplace(bytes, p);
  }
  void* stage(size_t bytes) {
    if (bytes > hStageBytes) {
      if (hStage) cudaFreeHost(hStage);
      hStage = nullptr;
      size_t nb = std::max<size_t>(bytes, hStageBytes * 2);
      CK(cudaMallocHost(&hStage, nb));
      hStageBytes = nb;
    }
    return hStage;
  }
};

BatchMem::~BatchMem() {
  if (!ctx) return;
  for (auto& b : blocks) ctx->dev_free(b.p);
}
void* BatchMem::alloc(size_t bytes) {
  void* p = ctx->dev_alloc(bytes);
  blocks.push_back({p, bytes});
  return p;
}

template <typename T>
T* dalloc(BatchMem& m, size_t count) {
  return static_cast<T*>(m.alloc(sizeof(T) * std::max<size_t>(count, 1)));
}

// Device bytes a TF may take: 160 per cluster (+ 48 with the compressed TF)
uint64_t footprint_of(uint64_t n, bool compress = false) {
  return (compress ? 208ull : 160ull) * n + (64ull << 20);
}

// Device layout of a host-resident TF's copy: the packed records, or
// sector[n] u8 | row[n] u8 | pad to 16 B | y[n] f32 | z[n] f32.
void input_layout(const o2tpc_tf& t, void* p, TFDesc& d) {
  if (t.format == O2TPC_FMT_FIXED) {
    d.in0 = p;
    return;
  }
  uint8_t* b = static_cast<uint8_t*>(p);
  float* py = reinterpret_cast<float*>(b + ((2 * t.n + 15) / 16) * 16);
  d.in0 = b;
  d.in1 = b + t.n;
  d.y = py;
  // the fourth array is z, or the drift time when the TF carries no z
  d.z = t.z ? py + t.n : nullptr;
  d.time = t.z ? nullptr : py + t.n;
}

void input_upload(const o2tpc_tf& t, void* p, cudaStream_t s) {
  TFDesc d{};
  input_layout(t, p, d);
  if (t.format == O2TPC_FMT_FIXED) {
    CK(cudaMemcpyAsync(p, t.packed, 12 * t.n, cudaMemcpyHostToDevice, s));
    return;
  }
  CK(cudaMemcpyAsync(const_cast<void*>(d.in0), t.sector, t.n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(const_cast<void*>(d.in1), t.row, t.n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(const_cast<float*>(d.y), t.y, 4 * t.n, cudaMemcpyHostToDevice, s));
  if (t.z) CK(cudaMemcpyAsync(const_cast<float*>(d.z), t.z, 4 * t.n, cudaMemcpyHostToDevice, s));
  else CK(cudaMemcpyAsync(const_cast<float*>(d.time), t.time, 4 * t.n, cudaMemcpyHostToDevice, s));
}

int read_int(Ctx* c, const int* dptr) {
  int v = 0;
  CK(cudaMemcpyAsync(&v, dptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return v;
}

// ------------------------------------------------------------ the batch
void tune_cache_store(Ctx* c);

// Autotuner: the cell sort and the NeighboursFinder are pure functions of
// their inputs, so every candidate launch shape is timed on the batch at hand
// (cell sort: best of two runs; CUDA events on the compute stream) and the fastest
// is kept for this and later batches.  The last cell-sort run leaves the same
// arrays as any other; the grid's block map is rebuilt for the chosen NF
// shape before the real NeighboursFinder launch.
void autotune(Ctx* c, int n, int nRows, const int* rowCnt, const int* rowMin, const int* rowMax, RowGrid* grid,
              int* nfBlockStart, int* totals, const int4* bucket, int* cellStart, int2* syz, int* sorig,
              int* gscratch, unsigned* err) {
  cudaStream_t st = c->stream;
  const GeomConst* G = c->dGeom;
  static const int kSort[3] = {128, 256, 512};
  static const int kNF[3] = {64, 128, 256};
  cudaEvent_t es[3][3], en[6][2];
  for (auto& r : es)
    for (auto& e : r) CK(cudaEventCreate(&e));
  for (auto& r : en)
    for (auto& e : r) CK(cudaEventCreate(&e));
  // scratch links for the timing runs of the NeighboursFinder
  int* up = static_cast<int*>(c->dev_alloc(sizeof(int) * (size_t)n * 2));
  for (int i = 0; i < 3; ++i) {
    CK(cudaEventRecord(es[i][0], st));
    launch_cell_sort(nRows, grid, bucket, cellStart, syz, sorig, gscratch, totals, st, kSort[i]);
    CK(cudaEventRecord(es[i][1], st));
    launch_cell_sort(nRows, grid, bucket, cellStart, syz, sorig, gscratch, totals, st, kSort[i]);
    CK(cudaEventRecord(es[i][2], st));
  }
  for (int i = 0; i < 6; ++i) {
    const int hb = kNF[i % 3];
    launch_grid(nRows, rowCnt, rowMin, rowMax, G, grid, nfBlockStart, hb, totals, st);
    const int blocks = n / hb + nRows + 1;
    CK(cudaEventRecord(en[i][0], st));
    launch_neighbours(blocks, hb, i >= 3, grid, nfBlockStart, nRows, cellStart, syz, G, up, up + n, err, st);
    CK(cudaEventRecord(en[i][1], st));
  }
  CK(cudaEventSynchronize(en[5][1]));
  c->dev_free(up);
  int bs = 0, bn = 0;
  for (int i = 0; i < 3; ++i) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, es[i][0], es[i][1]);
    cudaEventElapsedTime(&b, es[i][1], es[i][2]);
    c->tune.sort_ms[i] = std::min(a, b);
    if (c->tune.sort_ms[i] < c->tune.sort_ms[bs]) bs = i;
  }
  for (int i = 0; i < 6; ++i) {
    float m = 0.f;
    cudaEventElapsedTime(&m, en[i][0], en[i][1]);
    c->tune.nf_ms[i] = m;
    if (c->tune.nf_ms[i] < c->tune.nf_ms[bn]) bn = i;
  }
  for (auto& r : es)
    for (auto& e : r) cudaEventDestroy(e);
  for (auto& r : en)
    for (auto& e : r) cudaEventDestroy(e);
  c->tune.sort_threads_per_row = kSort[bs];
  c->tune.nf_hits_per_block = kNF[bn % 3];
  c->tune.nf_staged = bn >= 3 ? 1 : 0;
  c->tune.tuned = 1;
  c->tune.tuned_on_clusters = n;
  tune_cache_store(c);
  launch_grid(nRows, rowCnt, rowMin, rowMax, G, grid, nfBlockStart, c->tune.nf_hits_per_block, totals, st);
}

// What the download and the kept stages need from a pipeline run.
struct Pipe {
  int B = 0, n = 0, nHeads = 0;
  long long launches = 0;
  std::vector<TFDesc> tfd;
  const RowGrid* grid = nullptr;
  int *cellStart = nullptr, *sorig = nullptr, *upRaw = nullptr, *dnRaw = nullptr, *up = nullptr, *dn = nullptr;
  int* starts = nullptr;
  int2* syz = nullptr;
  TrackletBufs tb{};
  SectorTrackBufs sb{};
  MergeBufs mb{};
  OutBufs ob{};
  const int *trkTfBegin = nullptr, *stTfBegin = nullptr, *tlTfBegin = nullptr;
  const unsigned* dErr = nullptr;
  int graphSlot = 0;                 // captured path: the set of result arrays written
  std::shared_ptr<BatchMem> outMem;  // result arrays freed after the download (regular path)
  uint8_t* ctf = nullptr;            // compressed TFs of the batch, at ctfOff[i]
  std::vector<long long> ctfOff;
};

// A batch runs on the captured path when it fits the arena.
bool graph_fits(const Ctx* c, const std::vector<std::shared_ptr<Job>>& jobs) {
  if (c->cfg.flags & O2TPC_FLAG_COMPRESS) return false;  // the compressed TF reads its blob size back
  const GraphCaps& k = c->graph->caps;
  if ((int)jobs.size() > k.BCap) return false;
  long long n = 0, nc = 0;
  for (auto& j : jobs) {
    n += (long long)j->tf.n;
    nc += (long long)j->tf.n_coll;
  }
  return n <= k.nCap && nc <= k.collCap;
}

size_t r256(size_t x) { return (x + 255) / 256 * 256; }

// The captured path: the TF table, tiles and sizes are written into the
// arena, then one graph launch runs the whole pipeline (captured on first
// use, again after the launch shapes changed).  Returns false, with nothing
// for the caller to undo, when a capacity overflowed or the capture failed:
// the batch then runs on the regular path.
bool run_captured(Ctx* c, std::vector<std::shared_ptr<Job>>& jobs, BatchMem& M, Pipe& pp) {
  (void)M;
  GraphArena& A = *c->graph;
  const GraphCaps& k = A.caps;
  cudaStream_t st = c->stream;
  const int B = (int)jobs.size();
  std::vector<TFDesc> tfd(k.BCap);
  std::vector<int2> tiles;
  long long N = 0;
  size_t inOff = 0;
  int nColl = 0;
  for (int i = 0; i < B; ++i) {
    const o2tpc_tf& t = jobs[i]->tf;
    TFDesc d{};
    d.format = t.format;
    d.n = (int)t.n;
    d.inBase = (int)N;
    if (t.location == O2TPC_LOC_DEVICE || t.n == 0) {
      d.in0 = t.format == O2TPC_FMT_FIXED ? t.packed : (const void*)t.sector;
      d.in1 = t.row;
      d.y = t.y;
      d.z = t.z;
      d.time = t.time;
    } else if (jobs[i]->upState == 4) {  // uploaded ahead (the batch waited for the copy)
      input_layout(t, jobs[i]->dIn, d);
    } else {
      void* p = A.input + inOff;
      inOff += r256(input_bytes(t));
      input_upload(t, p, st);
      input_layout(t, p, d);
    }
    d.tileBase = (int)tiles.size();
    d.nTiles = (int)((t.n + k.tileSize - 1) / k.tileSize);
    for (int q = 0; q < d.nTiles; ++q) tiles.push_back(make_int2(i, q * k.tileSize));
    d.nColl = (int)t.n_coll;
    d.collBase = nColl;
    nColl += (int)t.n_coll;
    tfd[i] = d;
    N += (long long)t.n;
  }
  for (int i = B; i < k.BCap; ++i) {  // empty TFs up to the capacity
    TFDesc d{};
    d.format = O2TPC_FMT_FIXED;
    d.inBase = (int)N;
    d.in0 = A.input;
    d.tileBase = (int)tiles.size();
    tfd[i] = d;
  }
  while ((int)tiles.size() < k.nTilesCap) tiles.push_back(make_int2(0, 1 << 30));  // no clusters
  {
    Counts hc{};
    hc.n = (int)N;
    hc.nKeys = k.nKeys;
    const size_t b1 = sizeof(TFDesc) * k.BCap, b2 = sizeof(int2) * k.nTilesCap, b3 = sizeof(Counts);
    const size_t b4 = sizeof(double) * nColl;
    char* h = static_cast<char*>(c->stage(b1 + b2 + b3 + b4));
    memcpy(h, tfd.data(), b1);
    memcpy(h + b1, tiles.data(), b2);
    memcpy(h + b1 + b2, &hc, b3);
    for (int i = 0; i < B; ++i)
      if (tfd[i].nColl) memcpy(h + b1 + b2 + b3 + sizeof(double) * tfd[i].collBase, jobs[i]->tf.coll_time,
                               sizeof(double) * tfd[i].nColl);
    CK(cudaMemcpyAsync(A.tfs, h, b1, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(A.tiles, h + b1, b2, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(A.cnt, h + b1 + b2, b3, cudaMemcpyHostToDevice, st));
    if (nColl) CK(cudaMemcpyAsync(A.coll, h + b1 + b2 + b3, b4, cudaMemcpyHostToDevice, st));
  }
  // this replay writes result set `slot`, whose last results (two replays
  // back) must have reached the host first
  const int slot = c->graphSlot;
  if (c->graphDlRecorded[slot]) CK(cudaStreamWaitEvent(st, c->graphDl[slot], 0));
  if (c->graphExec[0] && (c->graphNf != c->tune.nf_hits_per_block * 2 + c->tune.nf_staged ||
                          c->graphSort != c->tune.sort_threads_per_row)) {
    for (auto& e : c->graphExec) {
      if (e) cudaGraphExecDestroy(e);
      e = nullptr;
    }
  }
  if (!c->graphExec[0]) {
    for (int s = 0; s < 2; ++s) {
      GraphArena As = A;
      if (s == 1) As.ob = A.ob2;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      const long long before = g_launch_count;
      graph_enqueue(As, c->dGeom, c->tune.nf_hits_per_block, c->tune.nf_staged != 0, c->tune.sort_threads_per_row,
                    (c->cfg.flags & O2TPC_FLAG_FORCE_FP64) ? 1 : 0, st,
                    (c->cfg.flags & O2TPC_FLAG_COOP_SEARCH) != 0, (c->cfg.flags & O2TPC_FLAG_ROW_STEP2) != 0);
      const cudaError_t ce = cudaStreamEndCapture(st, &g);
      c->graphKernels = g_launch_count - before;
      if (ce != cudaSuccess || !g || cudaGraphInstantiate(&c->graphExec[s], g, 0) != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        for (auto& e : c->graphExec) {
          if (e) cudaGraphExecDestroy(e);
          e = nullptr;
        }
        std::fprintf(stderr, "o2tpc: graph capture failed; batches run on the regular path\n");
        c->graph.reset();
        return false;
      }
      cudaGraphDestroy(g);
    }
    c->graphNf = c->tune.nf_hits_per_block * 2 + c->tune.nf_staged;
    c->graphSort = c->tune.sort_threads_per_row;
  }
  g_launch_count = c->graphKernels;
  CK(cudaEventRecord(c->evs[0], st));
  CK(cudaGraphLaunch(c->graphExec[slot], st));
  CK(cudaEventRecord(c->ev1, st));
  int hv[10];
  CK(cudaMemcpyAsync(hv, A.cnt, sizeof(Counts), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hv + 8, A.mb.pairCount, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hv + 9, A.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Counts hc;
  memcpy(&hc, hv, sizeof(Counts));
  if (hc.overflow || hv[8] > k.pairCap || (hv[9] & (kErrOverflow | kErrMembrane))) return false;
  tfd.resize(B);
  pp.B = B;
  pp.n = (int)N;
  pp.tfd = tfd;
  pp.grid = A.grid;
  pp.ob = slot ? A.ob2 : A.ob;
  pp.graphSlot = slot;
  c->graphSlot = slot ^ 1;
  pp.nHeads = hc.nHeads;
  pp.trkTfBegin = A.trkTfBegin;
  pp.stTfBegin = A.stTfBegin;
  pp.tlTfBegin = A.tlTfBegin;
  pp.dErr = A.err;
  pp.launches = c->graphKernels;
  return true;
}

// The regular path: sizes read back at four points, buffers allocated
// exactly (the batch's memory M), stage events recorded.
void run_regular(Ctx* c, std::vector<std::shared_ptr<Job>>& jobs, BatchMem& M, Pipe& pp) {
  cudaStream_t st = c->stream;
  const int B = (int)jobs.size();
  const int nRows = B * kRowsPerTF;
  // ---- inputs and TF table
  std::vector<TFDesc> tfd(B);
  std::vector<int2> tiles;
  long long N = 0;
  int nColl = 0;
  for (int i = 0; i < B; ++i) {
    const o2tpc_tf& t = jobs[i]->tf;
    TFDesc d{};
    d.format = t.format;
    d.n = (int)t.n;
    d.inBase = (int)N;
    if (t.location == O2TPC_LOC_DEVICE || t.n == 0) {
      d.in0 = t.format == O2TPC_FMT_FIXED ? t.packed : (const void*)t.sector;
      d.in1 = t.row;
      d.y = t.y;
      d.z = t.z;
      d.time = t.time;
    } else if (jobs[i]->upState == 4) {
      input_layout(t, jobs[i]->dIn, d);  // uploaded ahead on the copy stream
    } else {
      void* p = M.alloc(input_bytes(t));
      input_upload(t, p, st);
      input_layout(t, p, d);
    }
    int tileSize = std::max(kTileMin, (int)((t.n + kTilesPerTFMax - 1) / kTilesPerTFMax));
    d.tileBase = (int)tiles.size();
    d.nTiles = (int)((t.n + tileSize - 1) / tileSize);
    for (int k = 0; k < d.nTiles; ++k) tiles.push_back(make_int2(i, k * tileSize));
    d.nColl = (int)t.n_coll;
    d.collBase = nColl;
    nColl += (int)t.n_coll;
    tfd[i] = d;
    N += (long long)t.n;
  }
  // one tile size for the launch: the largest any TF asked for
  int tileSize = kTileMin;
  for (int i = 0; i < B; ++i) tileSize = std::max(tileSize, (int)((jobs[i]->tf.n + kTilesPerTFMax - 1) / kTilesPerTFMax));
  tiles.clear();
  for (int i = 0; i < B; ++i) {
    tfd[i].tileBase = (int)tiles.size();
    tfd[i].nTiles = (int)((jobs[i]->tf.n + tileSize - 1) / tileSize);
    for (int k = 0; k < tfd[i].nTiles; ++k) tiles.push_back(make_int2(i, k * tileSize));
  }
  const int nTiles = (int)tiles.size();
  const int n = (int)N;
  M.N = n;
  TFDesc* dTF = dalloc<TFDesc>(M, B);
  int2* dTiles = dalloc<int2>(M, nTiles);
  double* dColl = dalloc<double>(M, nColl);
  Counts* C = c->dCounts;  // device-side sizes of this batch (the context's own slot)
  {
    Counts hc{};
    hc.n = n;
    hc.nKeys = B * kNSec * 2;
    size_t b1 = sizeof(TFDesc) * B, b2 = sizeof(int2) * nTiles, b3 = sizeof(Counts), b4 = sizeof(double) * nColl;
    char* h = static_cast<char*>(c->stage(b1 + b2 + b3 + b4));
    memcpy(h, tfd.data(), b1);
    memcpy(h + b1, tiles.data(), b2);
    memcpy(h + b1 + b2, &hc, b3);
    for (int i = 0; i < B; ++i)
      if (tfd[i].nColl) memcpy(h + b1 + b2 + b3 + sizeof(double) * tfd[i].collBase, jobs[i]->tf.coll_time,
                               sizeof(double) * tfd[i].nColl);
    CK(cudaMemcpyAsync(dTF, h, b1, cudaMemcpyHostToDevice, st));
    if (nTiles) CK(cudaMemcpyAsync(dTiles, h + b1, b2, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(C, h + b1 + b2, b3, cudaMemcpyHostToDevice, st));
    if (nColl) CK(cudaMemcpyAsync(dColl, h + b1 + b2 + b3, b4, cudaMemcpyHostToDevice, st));
  }
  unsigned* dErr = dalloc<unsigned>(M, 4);
  CK(cudaMemsetAsync(dErr, 0, 16, st));
  const GeomConst* G = c->dGeom;

  // ---- A1-A4: ingest, row statistics, grid, sort
  CK(cudaEventRecord(c->evs[0], st));
  int* tileStats = dalloc<int>(M, (size_t)std::max(nTiles, 1) * 3 * kRowsPerTF);
  int* rowCnt = dalloc<int>(M, nRows);
  int* rowMin = dalloc<int>(M, nRows);
  int* rowMax = dalloc<int>(M, nRows);
  RowGrid* grid = dalloc<RowGrid>(M, nRows + 1);
  int* nfBlockStart = dalloc<int>(M, nRows + 1);
  int* totals = dalloc<int>(M, 4);
  launch_ingest_stats(dTF, dTiles, nTiles, tileSize, G, tileStats, dErr, st);
  CKL();
  launch_row_reduce(dTF, B, tileStats, rowCnt, rowMin, rowMax, st);
  CKL();
  launch_grid(nRows, rowCnt, rowMin, rowMax, G, grid, nfBlockStart, c->tune.nf_hits_per_block, totals, st);
  CKL();
  const long long cellsMax = (long long)n / kHitsPerCell + 46ll * nRows + 1;
  CK(cudaEventRecord(c->evs[1], st));
  int* cellStart = dalloc<int>(M, cellsMax + 1);
  int* gscratch = dalloc<int>(M, cellsMax);
  int4* bucket = dalloc<int4>(M, n);
  int2* syz = dalloc<int2>(M, (size_t)n + 2);  // padding read by the NeighboursFinder's aligned slab copies
  int* sorig = dalloc<int>(M, n);
  launch_row_scatter(dTF, dTiles, nTiles, tileSize, G, tileStats, grid, bucket, st);
  CKL();
  launch_cell_sort(nRows, grid, bucket, cellStart, syz, sorig, gscratch, totals, st, c->tune.sort_threads_per_row);
  if ((c->cfg.flags & O2TPC_FLAG_AUTOTUNE) && !c->tune.tuned && n >= (1 << 20))
    autotune(c, n, nRows, rowCnt, rowMin, rowMax, grid, nfBlockStart, totals, bucket, cellStart, syz, sorig, gscratch,
             dErr);
  CKL();

  // ---- A5-A7: neighbours, cleaner, start hits
  CK(cudaEventRecord(c->evs[2], st));
  int* upRaw = dalloc<int>(M, n);
  int* dnRaw = dalloc<int>(M, n);
  int* up = dalloc<int>(M, n);
  int* dn = dalloc<int>(M, n);
  int* flag = dalloc<int>(M, n + 1);
  int* scratch = dalloc<int>(M, scan_scratch_ints((long long)n + 8) + (nRows + 8) * 2 / 4096 + 64);
  const int nfB = c->tune.nf_hits_per_block;
  const int nfBlocksMax = n / nfB + nRows + 1;
  launch_neighbours(nfBlocksMax, nfB, c->tune.nf_staged != 0, grid, nfBlockStart, nRows, cellStart, syz, G, upRaw,
                    dnRaw, dErr, st, c->cfg.debug_inject);
  CKL();
  if (c->cfg.flags & O2TPC_FLAG_ROW_STEP2) {
    launch_neighbours_gap(n, &C->n, grid, nRows, cellStart, syz, G, upRaw, dnRaw, st);
    CKL();
  }
  CK(cudaEventRecord(c->evs[3], st));
  launch_clean(n, &C->n, upRaw, dnRaw, up, dn, flag, st);
  CKL();
  int* tileCnt = dalloc<int>(M, ballot_tiles(n) + 1);
  int* tileOff = dalloc<int>(M, ballot_tiles(n) + 1);
  launch_ballot_count(n, &C->n, flag, tileCnt, tileOff, &C->nTl, INT_MAX, &C->overflow, scratch, st);
  CKL();
  const int nTl = read_int(c, &C->nTl);  // sync 1
  M.nTl = nTl;
  int* starts = dalloc<int>(M, nTl);
  launch_ballot_compact(n, &C->n, flag, tileOff, starts, nTl, &C->overflow, st);
  CKL();
  int* tlTfBegin = dalloc<int>(M, B + 1);
  launch_tf_ranges(B, grid, starts, &C->nTl, tlTfBegin, st);
  CKL();

  // ---- A8: tracklets
  CK(cudaEventRecord(c->evs[4], st));
  TrackletBufs tb;
  tb.nhits = dalloc<int>(M, nTl + 1);
  tb.nasc = dalloc<int>(M, nTl);
  tb.hits = dalloc<int>(M, (size_t)nTl * kMaxTlHits);
  tb.rows = dalloc<uint8_t>(M, (size_t)nTl * kMaxTlHits);
  tb.state = dalloc<float>(M, (size_t)nTl * 21);
  tb.zref = dalloc<int>(M, nTl);
  tb.yref = dalloc<int>(M, nTl);
  tb.rbase = dalloc<int>(M, nTl);
  int* workCounter = dalloc<int>(M, 4);
  launch_tracklets(nTl, &C->nTl, workCounter, starts, up, grid, nRows, cellStart, syz, G, tb, st, c->evTl,
                   (c->cfg.flags & O2TPC_FLAG_COOP_SEARCH) != 0);
  CKL();

  // ---- A9: selection
  CK(cudaEventRecord(c->evs[5], st));
  unsigned long long* w = dalloc<unsigned long long>(M, n);
  CK(cudaMemsetAsync(w, 0, sizeof(unsigned long long) * std::max(n, 1), st));
  int* secBegin = dalloc<int>(M, B * kNSec + 1);
  int* wide = dalloc<int>(M, 1);
  launch_ownership(nTl, &C->nTl, B * kNSec, grid, starts, tb, w, secBegin, wide, st);
  CKL();
  int* nSeg = dalloc<int>(M, nTl + 1);
  int* nSegHits = dalloc<int>(M, nTl + 1);
  int* segPos = dalloc<int>(M, nTl + 1);
  int* segHitPos = dalloc<int>(M, nTl + 1);
  launch_segments_count(nTl, &C->nTl, secBegin, wide, w, tb, nSeg, nSegHits, st);
  CKL();
  scan_exclusive(nSeg, segPos, nTl, &C->nTl, scratch, st);
  CKL();
  scan_exclusive(nSegHits, segHitPos, nTl, &C->nTl, scratch, st);
  CKL();
  launch_count_at(segPos, &C->nTl, &C->nSt, INT_MAX, &C->overflow, st, segHitPos, &C->nStHits, INT_MAX);
  CKL();
  int hv[2];
  CK(cudaMemcpyAsync(hv, &C->nSt, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));  // sync 2
  const int nSt = hv[0], nStHits = hv[1];
  M.nSt = nSt;
  SectorTrackBufs sb;
  sb.tl = dalloc<int>(M, nSt);
  sb.sector = dalloc<int>(M, nSt);
  sb.tf = dalloc<int>(M, nSt);
  sb.zref = dalloc<int>(M, nSt);
  sb.off = dalloc<int>(M, nSt + 1);
  sb.hits = dalloc<int>(M, nStHits);
  sb.rows = dalloc<uint8_t>(M, nStHits);
  sb.yz = dalloc<int2>(M, nStHits);
  sb.orig = dalloc<int>(M, nStHits);
  sb.in = dalloc<float>(M, (size_t)nSt * 21);
  sb.out = dalloc<float>(M, (size_t)nSt * 21);
  launch_segments_write(nTl, &C->nTl, secBegin, wide, w, tb, segPos, segHitPos, syz, sorig, sb, nSt, nStHits, st);
  CKL();
  // CSR end: sb.off[nSt] = nStHits
  launch_count_at(segPos, &C->nTl, &C->nSt, nSt, &C->overflow, st, segHitPos, &C->nStHits, nStHits, sb.off);
  CKL();
  launch_st_gather(nStHits, &C->nStHits, sb, syz, sorig, st);
  CKL();
  CK(cudaEventRecord(c->evs[6], st));
  int* lenHist = dalloc<int>(M, kLenBins);
  int* stOrder = dalloc<int>(M, nSt);
  launch_len_order(nSt, &C->nSt, sb.off, lenHist, stOrder, st);
  launch_sector_fit(nSt, &C->nSt, tb, syz, G, sb, stOrder, st);
  CKL();
  int* stTfBegin = dalloc<int>(M, B + 1);
  int* tfKeys = dalloc<int>(M, B + 1);
  launch_iota(tfKeys, B + 1, st);
  launch_lower_bounds(sb.tf, &C->nSt, tfKeys, B + 1, stTfBegin, st);
  CKL();

  // ---- A10: merger
  CK(cudaEventRecord(c->evs[7], st));
  const int nKeys = B * kNSec * 2;
  MergeBufs mb;
  mb.nSt = nSt;
  mb.cnt = C;
  mb.keyIn = dalloc<int>(M, nSt);
  mb.keyOut = dalloc<int>(M, nSt);
  mb.listCnt = dalloc<int>(M, nKeys + 1);
  mb.listStart = dalloc<int>(M, nKeys + 1);
  mb.listItems = dalloc<int>(M, nSt);
  mb.listKey = dalloc<int>(M, nSt);
  mb.pairCount = dalloc<int>(M, 1);
  mb.edgeCnt = dalloc<int>(M, nKeys + 1);
  mb.edgeStart = dalloc<int>(M, nKeys + 1);
  mb.next = dalloc<int>(M, nSt);
  mb.prev = dalloc<int>(M, nSt);
  mb.reached = dalloc<int>(M, nSt);
  mb.pairCap = std::max(1024, 2 * nSt);
  mb.pairs = dalloc<float4>(M, mb.pairCap);
  mb.pairsSorted = dalloc<float4>(M, mb.pairCap);
  mb.sortScratch = dalloc<float4>(M, 2 * (size_t)std::max(mb.pairCap, nSt) + 16);
  launch_merge_keys(nSt, sb, G, mb, nKeys, scratch, st);
  CKL();
  launch_merge_pairs(nSt, sb, G, mb, dErr, st);
  CKL();
  int nPairs = read_int(c, mb.pairCount);  // sync 3
  if (nPairs > mb.pairCap) {
    mb.pairCap = nPairs + 1024;
    mb.pairs = dalloc<float4>(M, mb.pairCap);
    mb.pairsSorted = dalloc<float4>(M, mb.pairCap);
    mb.sortScratch = dalloc<float4>(M, 2 * (size_t)std::max(mb.pairCap, nSt) + 16);
    launch_merge_pairs(nSt, sb, G, mb, dErr, st);  // the overflow bit of the first pass is ignored
    nPairs = read_int(c, mb.pairCount);
  }
  launch_merge_select(nPairs, nKeys, mb, scratch, st);
  CKL();
  int* headFlag = dalloc<int>(M, nSt + 1);
  launch_chains(nSt, mb, headFlag, st);
  CKL();
  launch_ballot_count(nSt, &C->nSt, headFlag, tileCnt, tileOff, &C->nHeads, INT_MAX, &C->overflow, scratch, st);
  CKL();
  const int nHeads = read_int(c, &C->nHeads);  // sync 4
  int* heads = dalloc<int>(M, nHeads);
  launch_ballot_compact(nSt, &C->nSt, headFlag, tileOff, heads, nHeads, &C->overflow, st);
  CKL();

  // ---- A11: final refit and output
  CK(cudaEventRecord(c->evs[8], st));
  int* trkNcl = dalloc<int>(M, nHeads + 1);
  // result arrays live apart from the batch's other buffers: they stay until
  // the download stream has copied them out
  auto outMem = std::make_shared<BatchMem>();
  outMem->ctx = c;
  BatchMem& OM = *outMem;
  OutBufs ob;
  ob.off = dalloc<int>(OM, nHeads + 1);
  ob.cl = dalloc<int>(OM, nStHits);
  ob.x = dalloc<float>(OM, nHeads);
  ob.alpha = dalloc<float>(OM, nHeads);
  ob.par = dalloc<float>(OM, (size_t)nHeads * 5);
  ob.cov = dalloc<float>(OM, (size_t)nHeads * 15);
  ob.chi2 = dalloc<float>(OM, nHeads);
  ob.ndf = dalloc<int>(OM, nHeads);
  ob.sector = dalloc<uint8_t>(OM, nHeads);
  ob.flags = dalloc<uint8_t>(OM, nHeads);
  ob.zref = dalloc<int>(OM, nHeads);
  ob.nFallback = dalloc<int>(OM, 1);
  ob.fallback = dalloc<int>(M, nHeads);
  ob.ends = dalloc<int4>(M, nHeads);
  ob.endsR = dalloc<int2>(M, nHeads);
  ob.t0 = dalloc<float>(OM, nHeads);
  ob.t0err = dalloc<float>(OM, nHeads);
  ob.t0lo = dalloc<float>(OM, nHeads);
  ob.t0hi = dalloc<float>(OM, nHeads);
  ob.mate = dalloc<int>(OM, nHeads);
  ob.coll = dalloc<int>(OM, nHeads);
  CK(cudaMemsetAsync(ob.nFallback, 0, sizeof(int), st));
  launch_chain_counts(nHeads, &C->nHeads, heads, sb, mb, trkNcl, st);
  CKL();
  scan_exclusive(trkNcl, ob.off, nHeads, &C->nHeads, scratch, st);
  CKL();
  launch_final_refit(nHeads, &C->nHeads, heads, sb, mb, syz, sorig, dTF, G,
                     (c->cfg.flags & O2TPC_FLAG_FORCE_FP64) ? 1 : 0, ob, st);
  CKL();
  int* trkTfBegin = dalloc<int>(M, B + 1);
  launch_lower_bounds(heads, &C->nHeads, stTfBegin, B + 1, trkTfBegin, st);
  CKL();
  // ---- continuous readout: t0, membrane links, collision assignment
  CK(cudaEventRecord(c->evs[11], st));
  {
    // the merger's buffers, with links and a pair count of the stage's own
    MergeBufs mm = mb;
    mm.next = dalloc<int>(M, nHeads);
    mm.prev = dalloc<int>(M, nHeads);
    mm.pairCount = dalloc<int>(M, 1);
    launch_continuous(nHeads, &C->nHeads, nKeys, ob, mm, G, dTF, dColl, trkTfBegin, dErr, scratch, st);
  }
  CKL();
  // ---- compressed TF: hit removal, track model, rANS (one size read for the blob)
  if (c->cfg.flags & O2TPC_FLAG_COMPRESS) {
    CK(cudaEventRecord(c->evCtf[0], st));
    CtfBufs cb{};
    cb.nSeqCap = n;
    cb.nTrkCap = nHeads;
    cb.chunkCap = ctf_chunk_cap(n, nHeads, B);
    cb.onTrack = dalloc<uint8_t>(M, (size_t)n + 1);
    cb.firstFlag = dalloc<int>(M, (size_t)n + 1);
    cb.trkAtFirst = dalloc<int>(M, n);
    cb.unFlag = dalloc<int>(M, (size_t)n + 1);
    cb.canonFirst = dalloc<int>(M, nHeads);
    cb.canonTrk = dalloc<int>(M, nHeads);
    cb.len = dalloc<int>(M, (size_t)nHeads + 1);
    cb.lenScan = dalloc<int>(M, (size_t)nHeads + 1);
    cb.unList = dalloc<int>(M, n);
    cb.inBase = dalloc<int>(M, B + 1);
    cb.tfKt = dalloc<int>(M, B + 1);
    cb.tfUn = dalloc<int>(M, B + 1);
    cb.counts = dalloc<int>(M, 4);
    cb.tfCounts = dalloc<int>(M, 3 * B);
    cb.sd = dalloc<CtfStream>(M, 10 * B);
    cb.sym = dalloc<uint8_t>(M, 8 * (size_t)n + 2 * (size_t)nHeads + 16);
    cb.hist = dalloc<unsigned>(M, 2560 * (size_t)B);
    cb.freq = dalloc<uint16_t>(M, 2560 * (size_t)B);
    cb.enc = dalloc<uint2>(M, 2560 * (size_t)B);
    cb.degen = dalloc<int>(M, 10 * (size_t)B);
    cb.scratch = dalloc<uint8_t>(M, (size_t)cb.chunkCap * kCtfChunkBytes);
    cb.bytes = dalloc<int>(M, (size_t)cb.chunkCap + 1);
    cb.payOff = dalloc<int>(M, (size_t)cb.chunkCap + 1);
    cb.tfBlob = dalloc<long long>(M, B + 1);
    cb.tfHead = dalloc<long long>(M, B);
    launch_ctf_symbols(n, &C->n, nHeads, &C->nHeads, B, dTF, grid, nRows, syz, sorig, heads, sb, mb, ob, cb, tileCnt,
                       tileOff, &C->overflow, scratch, st);
    CKL();
    pp.ctfOff.resize(B + 1);
    CK(cudaMemcpyAsync(pp.ctfOff.data(), cb.tfBlob, sizeof(long long) * (B + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));  // sync 5
    pp.ctf = dalloc<uint8_t>(OM, (size_t)pp.ctfOff[B] + 16);
    launch_ctf_blob(B, cb, pp.ctf, st);
    CKL();
    CK(cudaEventRecord(c->evCtf[1], st));
  }
  CK(cudaEventRecord(c->ev1, st));
  CK(cudaEventRecord(c->evs[9], st));

  pp.B = B;
  pp.n = n;
  pp.tfd = tfd;
  pp.grid = grid;
  pp.cellStart = cellStart;
  pp.sorig = sorig;
  pp.syz = syz;
  pp.upRaw = upRaw;
  pp.dnRaw = dnRaw;
  pp.up = up;
  pp.dn = dn;
  pp.starts = starts;
  pp.tb = tb;
  pp.sb = sb;
  pp.mb = mb;
  pp.ob = ob;
  pp.nHeads = nHeads;
  pp.trkTfBegin = trkTfBegin;
  pp.stTfBegin = stTfBegin;
  pp.tlTfBegin = tlTfBegin;
  pp.dErr = dErr;
  pp.outMem = outMem;
  pp.launches = g_launch_count;
}

// Autotuner cache: one line per GPU model, "<name>\t<nf hits>\t<staged>\t<sort threads>".
std::string gpu_name(int dev) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n = p.name;
  for (auto& ch : n)
    if (ch == '\t' || ch == '\n') ch = ' ';
  return n;
}

void tune_cache_load(Ctx* c) {
  if (!c->cfg.tune_cache_path) return;
  FILE* f = std::fopen(c->cfg.tune_cache_path, "r");
  if (!f) return;
  const std::string me = gpu_name(c->cfg.device);
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    int nf = 0, staged = 0, sort = 0;
    if (me != line || std::sscanf(tab + 1, "%d %d %d", &nf, &staged, &sort) != 3) continue;
    if ((nf == 64 || nf == 128 || nf == 256) && (sort == 128 || sort == 256 || sort == 512)) {
      c->tune.nf_hits_per_block = nf;
      c->tune.nf_staged = staged ? 1 : 0;
      c->tune.sort_threads_per_row = sort;
      c->tune.tuned = 1;
    }
  }
  std::fclose(f);
}

void tune_cache_store(Ctx* c) {
  if (!c->cfg.tune_cache_path) return;
  const std::string me = gpu_name(c->cfg.device);
  std::vector<std::string> keep;
  if (FILE* f = std::fopen(c->cfg.tune_cache_path, "r")) {  // other GPU models' lines stay
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
      const char* tab = std::strchr(line, '\t');
      if (tab && std::string(line, (size_t)(tab - line)) != me) keep.emplace_back(line);
    }
    std::fclose(f);
  }
  FILE* f = std::fopen(c->cfg.tune_cache_path, "w");
  if (!f) return;
  for (auto& l : keep) std::fputs(l.c_str(), f);
  std::fprintf(f, "%s\t%d %d %d\n", me.c_str(), c->tune.nf_hits_per_block, c->tune.nf_staged,
               c->tune.sort_threads_per_row);
  std::fclose(f);
}

void run_batch(Ctx* c, std::vector<std::shared_ptr<Job>>& jobs) {
  cudaStream_t st = c->stream;
  const bool keep = (c->cfg.flags & O2TPC_FLAG_KEEP_STAGES) != 0;
  auto mem = std::make_shared<BatchMem>();
  mem->ctx = c;
  BatchMem& M = *mem;
  const int B = (int)jobs.size();
  const int nRows = B * kRowsPerTF;
  M.nTF = B;
  M.nRows = nRows;
  CK(cudaEventRecord(c->ev0, st));
  cudaEvent_t trS = nullptr, trE = nullptr;
  if (c->traceMode == 2) {
    CK(cudaEventCreate(&trS));
    CK(cudaEventCreate(&trE));
    CK(cudaEventRecord(trS, st));
  }
  const double hS = now_ms();
  g_launch_count = 0;
  // inputs uploaded ahead: the batch waits for their copies and owns their memory
  for (auto& jp : jobs) {
    if (jp->upState != 2) continue;
    M.blocks.push_back({jp->dIn, (size_t)jp->dInBytes});
    jp->upState = 4;  // the batch owns the copy now
    CK(cudaStreamWaitEvent(st, jp->upEv, 0));
    cudaEventDestroy(jp->upEv);
    jp->upEv = nullptr;
  }
  CK(cudaEventRecord(c->evWait, st));
  Pipe pp;
  bool captured = false;
  // a batch the autotuner still waits for runs on the regular path (the
  // graph is captured afterwards with the chosen shapes)
  long long nb = 0;
  for (auto& j : jobs) nb += (long long)j->tf.n;
  const bool tunePending = (c->cfg.flags & O2TPC_FLAG_AUTOTUNE) && !c->tune.tuned && nb >= (1 << 20);
  if (c->graph && !keep && !tunePending && graph_fits(c, jobs)) captured = run_captured(c, jobs, M, pp);
  if (!captured) run_regular(c, jobs, M, pp);

  // ---- A12: download.  Sizes first (synchronously), then every TF's arrays
  // straight into its own pinned result block on the download stream, which
  // the finisher thread waits for while the worker starts the next batch.
  const int n = pp.n, nHeads = pp.nHeads;
  const OutBufs& ob = pp.ob;
  const std::vector<TFDesc>& tfd = pp.tfd;
  const RowGrid* grid = pp.grid;
  const int *trkTfBegin = pp.trkTfBegin, *stTfBegin = pp.stTfBegin, *tlTfBegin = pp.tlTfBegin;
  const unsigned* dErr = pp.dErr;
  const size_t nT = (size_t)nHeads;
  int* hSmall = static_cast<int*>(c->stage(sizeof(int) * (nT + 1 + 3 * (B + 1) + 8)));
  int* hOff = hSmall;
  int* hTrkTf = hOff + nT + 1;
  int* hStTf = hTrkTf + B + 1;
  int* hTlTf = hStTf + B + 1;
  unsigned* hErr = reinterpret_cast<unsigned*>(hTlTf + B + 1);
  if (trE) CK(cudaEventRecord(trE, st));
  CK(cudaMemcpyAsync(hOff, ob.off, sizeof(int) * (nT + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hTrkTf, trkTfBegin, sizeof(int) * (B + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hStTf, stTfBegin, sizeof(int) * (B + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hTlTf, tlTfBegin, sizeof(int) * (B + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hErr, dErr, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  std::vector<RowGrid> tfFirstRow(B);
  for (int i = 0; i < B; ++i) CK(cudaMemcpyAsync(&tfFirstRow[i], grid + (size_t)i * kRowsPerTF, sizeof(RowGrid),
                                                 cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(c->evs[10], st));
  launch_stream_tail(st);
  CK(cudaStreamSynchronize(st));

  auto P = std::make_shared<Pending>();
  P->jobs = jobs;
  P->out = pp.outMem;
  P->captured = captured;
  P->trS = trS;
  P->trE = trE;
  P->hS = hS - c->hostRef;
  if (!captured) {  // the captured path records no stage events
    for (int k = 0; k < 10; ++k) cudaEventElapsedTime(&P->stageMs[k], c->evs[k], c->evs[k + 1]);
    // evs[11] splits step 8: the final refit, then the continuous-readout step
    cudaEventElapsedTime(&P->stageMs[8], c->evs[8], c->evs[11]);
    cudaEventElapsedTime(&P->stageMs[16], c->evs[11], (c->cfg.flags & O2TPC_FLAG_COMPRESS) ? c->evCtf[0] : c->evs[9]);
    if (c->cfg.flags & O2TPC_FLAG_COMPRESS) cudaEventElapsedTime(&P->stageMs[17], c->evCtf[0], c->evCtf[1]);
    cudaEventElapsedTime(&P->stageMs[12], c->evWait, c->evs[0]);
    cudaEventElapsedTime(&P->stageMs[14], c->evTl[0], c->evTl[1]);
    cudaEventElapsedTime(&P->stageMs[15], c->evTl[2], c->evTl[3]);
  }
  cudaEventElapsedTime(&P->stageMs[13], c->ev0, c->evWait);
  float devMs = 0.f;
  cudaEventElapsedTime(&devMs, c->ev0, c->ev1);
  const long long nLaunch = pp.launches;
  const bool inputBad = (*hErr & kErrInput) != 0;
  // more membrane candidate pairs than the buffer holds (2 per sector track):
  // the links would be incomplete, so the batch's TFs report ETOOBIG
  const bool memOverflow = (*hErr & kErrMembrane) != 0;
  const uint32_t events = (*hErr & kErrTimeout) ? 1u : 0u;
  cudaStream_t dl = c->dlStream;
  CK(cudaEventCreate(&P->dl0));
  CK(cudaEventCreate(&P->dl1));
  CK(cudaStreamWaitEvent(dl, c->evs[10], 0));
  CK(cudaEventRecord(P->dl0, dl));

  auto r16 = [](size_t x) { return (x + 15) / 16 * 16; };
  const double tPrep = now_ms();
  for (int i = 0; i < B; ++i) {
    Job& J = *jobs[i];
    const int t0 = hTrkTf[i], t1 = hTrkTf[i + 1];
    const size_t nt = (size_t)(t1 - t0);
    const size_t ncl = (size_t)(hOff[t1] - hOff[t0]);
    const size_t nctf = pp.ctf ? (size_t)(pp.ctfOff[i + 1] - pp.ctfOff[i]) : 0;
    const size_t bytes = r16(8 * (nt + 1)) + r16(4 * ncl) + 11 * r16(4 * nt) + r16(20 * nt) + r16(60 * nt) +
                         2 * r16(nt) + r16(nctf) + 64;
    J.host = c->pinned_get(bytes, &J.hostBytes);
    char* q = static_cast<char*>(J.host);
    auto take = [&](const void* dsrc, size_t nb) -> char* {
      char* dst = q;
      if (nb) {
        if (c->traceCopies && c->traceMode == 1) {
          cudaEvent_t a, b;
          cudaEventCreate(&a);
          cudaEventCreate(&b);
          cudaEventRecord(a, dl);
          CK(cudaMemcpyAsync(dst, dsrc, nb, cudaMemcpyDeviceToHost, dl));
          cudaEventRecord(b, dl);
          cudaEventSynchronize(b);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, a, b);
          std::fprintf(stderr, "o2tpc copy %zu bytes %.3f ms %.1f GB/s\n", nb, ms, nb / (ms * 1e6));
          cudaEventDestroy(a);
          cudaEventDestroy(b);
        } else {
          CK(cudaMemcpyAsync(dst, dsrc, nb, cudaMemcpyDeviceToHost, dl));
        }
      }
      q += r16(nb);
      return dst;
    };
    uint64_t* off64 = reinterpret_cast<uint64_t*>(q);
    q += r16(8 * (nt + 1));
    o2tpc_result& R = J.res;
    R.n_tracks = (uint64_t)nt;
    R.offsets = off64;
    R.cluster_idx = reinterpret_cast<const uint32_t*>(take(ob.cl + hOff[t0], 4 * ncl));
    R.x = reinterpret_cast<const float*>(take(ob.x + t0, 4 * nt));
    R.alpha = reinterpret_cast<const float*>(take(ob.alpha + t0, 4 * nt));
    R.par = reinterpret_cast<const float*>(take(ob.par + 5 * (size_t)t0, 20 * nt));
    R.cov = reinterpret_cast<const float*>(take(ob.cov + 15 * (size_t)t0, 60 * nt));
    R.chi2 = reinterpret_cast<const float*>(take(ob.chi2 + t0, 4 * nt));
    R.ndf = reinterpret_cast<const int32_t*>(take(ob.ndf + t0, 4 * nt));
    R.zeta_ref = reinterpret_cast<const uint32_t*>(take(ob.zref + t0, 4 * nt));
    R.sector = reinterpret_cast<const uint8_t*>(take(ob.sector + t0, nt));
    R.flags = reinterpret_cast<const uint8_t*>(take(ob.flags + t0, nt));
    R.t0 = reinterpret_cast<const float*>(take(ob.t0 + t0, 4 * nt));
    R.t0_err = reinterpret_cast<const float*>(take(ob.t0err + t0, 4 * nt));
    R.t0_lo = reinterpret_cast<const float*>(take(ob.t0lo + t0, 4 * nt));
    R.t0_hi = reinterpret_cast<const float*>(take(ob.t0hi + t0, 4 * nt));
    R.mate = reinterpret_cast<const int32_t*>(take(ob.mate + t0, 4 * nt));
    R.collision = reinterpret_cast<const int32_t*>(take(ob.coll + t0, 4 * nt));
    R.ctf = nctf ? reinterpret_cast<const uint8_t*>(take(pp.ctf + pp.ctfOff[i], nctf)) : nullptr;
    R.ctf_bytes = (uint64_t)nctf;
    for (size_t k = 0; k <= nt; ++k) off64[k] = (uint64_t)(hOff[t0 + k] - hOff[t0]);
    R.user_tag = J.tf.user_tag;
    R.stats.n_clusters = J.tf.n;
    R.stats.n_tracklets = (uint64_t)(hTlTf[i + 1] - hTlTf[i]);
    R.stats.n_sector_tracks = (uint64_t)(hStTf[i + 1] - hStTf[i]);
    R.stats.n_tracks = R.n_tracks;
    R.stats.batch_size = (uint32_t)B;
    R.stats.ms_queue = (float)(J.t_start - J.t_submit);
    R.stats.ms_device = devMs;
    R.stats.n_launches = (uint64_t)nLaunch;
    R.stats.events = events;
    J.status = inputBad ? O2TPC_EINVAL : (memOverflow ? O2TPC_ETOOBIG : O2TPC_OK);
    R.status = J.status;
    J.tfIndex = i;
  }
  CK(cudaEventRecord(P->dl1, dl));
  if (captured) {  // the replay after next writes these result arrays again
    CK(cudaEventRecord(c->graphDl[pp.graphSlot], dl));
    c->graphDlRecorded[pp.graphSlot] = true;
  }
  P->hostPrepMs = now_ms() - tPrep;
  P->hD = now_ms() - c->hostRef;

  M.tfHitBase.resize(B);
  M.tfHitEnd.resize(B);
  M.tfInBase.resize(B);
  M.tfTlBegin.assign(hTlTf, hTlTf + B + 1);
  M.tfStBegin.assign(hStTf, hStTf + B + 1);
  for (int i = 0; i < B; ++i) {
    M.tfHitBase[i] = tfFirstRow[i].start;
    M.tfHitEnd[i] = (i + 1 < B) ? tfFirstRow[i + 1].start : n;
    M.tfInBase[i] = tfd[i].inBase;
  }
  if (keep) {
    M.grid = const_cast<RowGrid*>(pp.grid);
    M.cellStart = pp.cellStart;
    M.sorig = pp.sorig;
    M.syz = pp.syz;
    M.upRaw = pp.upRaw;
    M.dnRaw = pp.dnRaw;
    M.up = pp.up;
    M.dn = pp.dn;
    M.starts = pp.starts;
    M.tb = pp.tb;
    M.sb = pp.sb;
    M.mb = pp.mb;
    M.refs = B;
    for (int i = 0; i < B; ++i) jobs[i]->mem = mem;
  }
  // hand the batch to the finisher; nothing below may throw
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->finQueue.push_back(P);
  }
  c->cvFin.notify_one();
  // without kept stages the batch memory is freed here (stream-ordered)
}

// Frees an upload made ahead that no batch took over (failed batch, destroy).
void release_upload(Ctx* c, Job& j) {
  if (j.upState != 2) return;
  if (j.upEv) {
    cudaEventSynchronize(j.upEv);
    cudaEventDestroy(j.upEv);
    j.upEv = nullptr;
  }
  c->dev_free(j.dIn);
  j.dIn = nullptr;
  j.upState = 3;
}

// Copy thread: uploads host-resident TFs that wait in the queue on the copy
// stream, so that their H2D transfer overlaps the batch computing before
// them (within upAheadLimit bytes of device memory).  Only with the
// library's own memory pool: a user allocator hands out memory that is
// ordered on the compute stream alone.
void uploader_main(Ctx* c) {
  cudaSetDevice(c->cfg.device);
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      c->cvUp.wait(lk, [&] {
        if (c->stop) return true;
        for (auto& q : c->queue) {
          if (q->upState != 0 || q->tf.location != O2TPC_LOC_HOST || q->tf.n == 0) continue;
          if (c->upAheadBytes + input_bytes(q->tf) > c->upAheadLimit) return false;  // keep queue order
          j = q;
          return true;
        }
        return false;
      });
      if (c->stop) return;
      j->upState = 1;
      j->dInBytes = input_bytes(j->tf);
      c->upAheadBytes += j->dInBytes;
    }
    bool ok = true;
    try {
      j->dIn = c->dev_alloc_on(j->dInBytes, c->upStream);
      input_upload(j->tf, j->dIn, c->upStream);
      CK(cudaEventCreateWithFlags(&j->upEv, cudaEventDisableTiming));
      CK(cudaEventRecord(j->upEv, c->upStream));
    } catch (...) {
      ok = false;
    }
    if (!ok) {
      cudaGetLastError();
      // memory not given back here stays with the copy stream until it drains
      if (j->upEv) cudaEventDestroy(j->upEv);
      j->upEv = nullptr;
      if (j->dIn) {
        cudaStreamSynchronize(c->upStream);
        c->dev_free(j->dIn);
        j->dIn = nullptr;
      }
    }
    {
      std::lock_guard<std::mutex> lk(c->mu);
      j->upState = ok ? 2 : 3;
      if (!ok) c->upAheadBytes -= j->dInBytes;
    }
    c->cvUp.notify_all();
  }
}

void worker_main(Ctx* c) {
  cudaSetDevice(c->cfg.device);
  for (;;) {
    std::vector<std::shared_ptr<Job>> batch;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      c->cvWork.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      if (c->queue.empty() && c->stop) return;
      uint64_t fp = 0, hits = 0;
      const int maxB = (c->cfg.flags & O2TPC_FLAG_NO_BATCHING) ? 1 : c->cfg.max_batch;
      while (!c->queue.empty() && (int)batch.size() < maxB) {
        auto& j = c->queue.front();
        // a TF joins only if the batch stays within the size that fills the
        // GPU: small TFs share batches, a large one runs alone and never
        // holds small ones back (FIFO order kept: stop at the first misfit)
        const uint64_t maxHits = (c->cfg.flags & O2TPC_FLAG_COMPRESS) ? kMaxCompressHits : kMaxBatchHits;
        if (!batch.empty() && (fp + j->footprint > c->cfg.mem_budget || hits + j->tf.n > maxHits ||
                               hits + j->tf.n > c->cfg.batch_full_clusters))
          break;
        // with a captured path, batches stay within its arena where they can
        if (!batch.empty() && c->graph &&
            ((int)batch.size() >= c->graph->caps.BCap || hits + j->tf.n > (uint64_t)c->graph->caps.nCap))
          break;
        fp += j->footprint;
        hits += j->tf.n;
        batch.push_back(j);
        c->queue.pop_front();
      }
      // a TF whose upload the copy thread is issuing right now is waited for;
      // the rest are left to the batch's stream
      c->cvUp.wait(lk, [&] {
        for (auto& j : batch)
          if (j->upState == 1) return false;
        return true;
      });
      for (auto& j : batch) {
        if (j->upState == 2) c->upAheadBytes -= j->dInBytes;
        else if (j->upState == 0) j->upState = 3;
      }
    }
    c->cvUp.notify_all();
    const double t0 = now_ms();
    for (auto& j : batch) j->t_start = t0;
    int status = O2TPC_OK;
    if (c->fatal != O2TPC_OK) {
      status = c->fatal;
    } else {
      try {
        run_batch(c, batch);
      } catch (const CudaError& e) {
        std::fprintf(stderr, "o2tpc: CUDA error %s at o2tpc_capi.cu:%d\n", cudaGetErrorString(e.e), e.line);
        cudaGetLastError();
        status = O2TPC_ECUDA;
        c->fatal = O2TPC_ECUDA;
      } catch (const AllocError&) {
        status = O2TPC_ENOMEM;
      } catch (const std::bad_alloc&) {
        status = O2TPC_ENOMEM;
      }
    }
    for (auto& j : batch) release_upload(c, *j);
    if (status == O2TPC_OK) continue;  // the finisher completes the batch
    {
      std::lock_guard<std::mutex> lk(c->mu);
      for (auto& j : batch) {
        j->status = status;
        j->res = o2tpc_result{};
        j->res.status = status;
        j->res.user_tag = j->tf.user_tag;
        j->emptyOffset = 0;
        j->res.offsets = &j->emptyOffset;
        j->t_end = now_ms();
        j->done = true;
      }
    }
    c->cvDone.notify_all();
  }
}

// Finisher: completes batches in order once their download has landed, then
// frees their device result arrays.
void finisher_main(Ctx* c) {
  cudaSetDevice(c->cfg.device);
  for (;;) {
    std::shared_ptr<Pending> P;
    {
      std::unique_lock<std::mutex> lk(c->mu);
      c->cvFin.wait(lk, [&] { return c->finStop || !c->finQueue.empty(); });
      if (c->finQueue.empty()) return;
      P = c->finQueue.front();
      c->finQueue.pop_front();
    }
    const cudaError_t e = cudaEventSynchronize(P->dl1);
    float dlMs = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&dlMs, P->dl0, P->dl1);
    if (e == cudaSuccess && P->trS && c->evRef) {
      float a = 0.f, b = 0.f, d0 = 0.f, d1 = 0.f;
      cudaEventElapsedTime(&a, c->evRef, P->trS);
      cudaEventElapsedTime(&b, c->evRef, P->trE);
      cudaEventElapsedTime(&d0, c->evRef, P->dl0);
      cudaEventElapsedTime(&d1, c->evRef, P->dl1);
      std::fprintf(stderr,
                   "o2tpc timeline: batch start %.3f compute end %.3f download %.3f - %.3f ms (host: start %.3f, "
                   "downloads issued %.3f, done seen %.3f)\n",
                   a, b, d0, d1, P->hS, P->hD, now_ms() - c->hostRef);
    }
    const double tEnd = now_ms();
    P->out.reset();
    if (e == cudaSuccess) {
      for (auto& jp : P->jobs) {
        o2tpc_result& R = jp->res;
        uint64_t fb = 0;
        for (uint64_t k = 0; k < R.n_tracks; ++k) fb += (R.flags[k] & 1) ? 1 : 0;
        R.stats.n_fp64_fallback = fb;
        for (int k = 0; k < 18; ++k) R.stats.ms_stage[k] = P->stageMs[k];
        R.stats.ms_stage[10] = dlMs;
        R.stats.ms_stage[11] = (float)P->hostPrepMs;
        R.stats.captured = P->captured ? 1u : 0u;
        R.stats.ms_batch = (float)(tEnd - jp->t_start);
      }
    } else {
      std::fprintf(stderr, "o2tpc: CUDA error %s in the result download\n", cudaGetErrorString(e));
      cudaGetLastError();
    }
    {
      std::lock_guard<std::mutex> lk(c->mu);
      if (e != cudaSuccess) c->fatal = O2TPC_ECUDA;
      for (auto& jp : P->jobs) {
        if (e != cudaSuccess) {
          jp->status = O2TPC_ECUDA;
          jp->res.status = O2TPC_ECUDA;
        }
        jp->t_end = tEnd;
        jp->done = true;
      }
    }
    c->cvDone.notify_all();
  }
}

}  // namespace

// =================================================================== C-ABI
extern "C" {

const char* o2tpc_strerror(int32_t s) {
  switch (s) {
    case O2TPC_OK: return "ok";
    case O2TPC_PENDING: return "pending";
    case O2TPC_EINVAL: return "invalid argument or cluster content";
    case O2TPC_ENOMEM: return "out of memory";
    case O2TPC_EAGAIN: return "queue full, retry later";
    case O2TPC_ETOOBIG: return "time frame exceeds the memory budget";
    case O2TPC_ECUDA: return "CUDA error";
    case O2TPC_ETIMEOUT: return "device wait timed out";
    case O2TPC_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

int o2tpc_create(const o2tpc_config* cfg, o2tpc_ctx** out) {
  if (!out) return O2TPC_EINVAL;
  *out = nullptr;
  o2tpc_config c{};
  c.bz_tesla = 0.5;
  c.vdrift_cm_us = 2.58;
  if (cfg) c = *cfg;
  if (c.mem_budget == 0) c.mem_budget = 120ull << 30;
  if (c.max_inflight <= 0) c.max_inflight = 64;
  if (c.max_batch <= 0) c.max_batch = 64;
  if (c.batch_full_clusters == 0) c.batch_full_clusters = kBatchFullHits;
  if (c.nf_hits_per_block == 0) c.nf_hits_per_block = kNFBlock;
  if (c.sort_threads_per_row == 0) c.sort_threads_per_row = 256;
  if ((c.nf_hits_per_block != 64 && c.nf_hits_per_block != 128 && c.nf_hits_per_block != 256) ||
      (c.sort_threads_per_row != 128 && c.sort_threads_per_row != 256 && c.sort_threads_per_row != 512))
    return O2TPC_EINVAL;
  if (!(c.vdrift_cm_us > 0.0) || !std::isfinite(c.bz_tesla)) return O2TPC_EINVAL;
  if ((c.dev_alloc == nullptr) != (c.dev_free == nullptr)) return O2TPC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
    cudaGetLastError();
    return O2TPC_ECUDA;
  }
  auto* x = new (std::nothrow) Ctx();
  if (!x) return O2TPC_ENOMEM;
  x->cfg = c;
  x->tune.nf_hits_per_block = c.nf_hits_per_block;
  x->tune.sort_threads_per_row = c.sort_threads_per_row;
  x->tune.nf_staged = c.nf_staged ? 1 : 0;
  if (c.flags & O2TPC_FLAG_AUTOTUNE) tune_cache_load(x);
  x->traceCopies = std::getenv("O2TPC_TRACE_COPIES") != nullptr;
  x->traceMode = x->traceCopies ? std::atoi(std::getenv("O2TPC_TRACE_COPIES")) : 0;
  try {
    CK(cudaSetDevice(c.device));
    if (c.stream) {
      x->stream = static_cast<cudaStream_t>(c.stream);
    } else {
      CK(cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking));
      x->ownStream = true;
    }
    CK(cudaEventCreate(&x->ev0));
    CK(cudaEventCreate(&x->ev1));
    CK(cudaEventCreate(&x->evWait));
    CK(cudaStreamCreateWithFlags(&x->upStream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&x->dlStream, cudaStreamNonBlocking));
    if (!c.dev_alloc) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = c.device;
      CK(cudaMemPoolCreate(&x->pool, &props));
      // keep freed memory for the next batch; never make the copy stream wait
      // for the compute stream to reuse a block
      uint64_t keepAll = ~0ull;
      int noInternalDeps = 0;
      CK(cudaMemPoolSetAttribute(x->pool, cudaMemPoolAttrReleaseThreshold, &keepAll));
      CK(cudaMemPoolSetAttribute(x->pool, cudaMemPoolReuseAllowInternalDependencies, &noInternalDeps));
      x->upAheadLimit = c.mem_budget / 8;
    }
    for (auto& e : x->evs) CK(cudaEventCreate(&e));
    if (x->traceMode == 2) {
      CK(cudaEventCreate(&x->evRef));
      CK(cudaEventRecord(x->evRef, x->stream));
      CK(cudaEventSynchronize(x->evRef));
      x->hostRef = now_ms();
    }
    for (auto& e : x->evTl) CK(cudaEventCreate(&e));
    for (auto& e : x->evCtf) CK(cudaEventCreate(&e));
    fill_geom(x->hGeom, c.bz_tesla, c.vdrift_cm_us);
    x->hGeom.angErr = (c.flags & O2TPC_FLAG_ANGULAR_ERRORS) ? 1 : 0;
    x->hGeom.rowStep2 = (c.flags & O2TPC_FLAG_ROW_STEP2) ? 1 : 0;
    x->dGeom = static_cast<GeomConst*>(x->dev_alloc(sizeof(GeomConst)));
    x->dCounts = static_cast<Counts*>(x->dev_alloc(sizeof(Counts)));
    CK(cudaMemcpyAsync(x->dGeom, &x->hGeom, sizeof(GeomConst), cudaMemcpyHostToDevice, x->stream));
    CK(cudaStreamSynchronize(x->stream));
  } catch (const CudaError&) {
    cudaGetLastError();
    delete x;
    return O2TPC_ECUDA;
  } catch (const AllocError&) {
    delete x;
    return O2TPC_ENOMEM;
  }
  if (c.graph_max_clusters > 0) {
    try {
      for (auto& e : x->graphDl) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      x->graph.reset(new GraphArena());
      x->graph->caps = graph_caps((long long)std::min<uint64_t>(c.graph_max_clusters, kMaxBatchHits / 2),
                                  c.graph_max_tfs > 0 ? c.graph_max_tfs : 64,
                                  (c.flags & O2TPC_FLAG_GRAPH_TIGHT) != 0);
      const size_t bytes = graph_carve(*x->graph, nullptr);
      x->graphMem = x->dev_alloc(bytes);
      graph_carve(*x->graph, static_cast<char*>(x->graphMem));
    } catch (...) {
      cudaGetLastError();
      x->graph.reset();
      o2tpc_destroy(reinterpret_cast<o2tpc_ctx*>(x));
      return O2TPC_ENOMEM;
    }
  }
  x->worker = std::thread(worker_main, x);
  x->finisher = std::thread(finisher_main, x);
  if (x->pool) x->uploader = std::thread(uploader_main, x);
  *out = reinterpret_cast<o2tpc_ctx*>(x);
  return O2TPC_OK;
}

static int check_tf(const Ctx* c, const o2tpc_tf* tf) {
  if (tf->format != O2TPC_FMT_FLOAT && tf->format != O2TPC_FMT_FIXED) return O2TPC_EINVAL;
  if (tf->location != O2TPC_LOC_HOST && tf->location != O2TPC_LOC_DEVICE) return O2TPC_EINVAL;
  if (tf->n > 0) {
    if (tf->format == O2TPC_FMT_FIXED && !tf->packed) return O2TPC_EINVAL;
    if (tf->format == O2TPC_FMT_FLOAT && (!tf->sector || !tf->row || !tf->y || (!tf->z && !tf->time)))
      return O2TPC_EINVAL;
  }
  if (tf->n_coll > 0) {
    if (!tf->coll_time || tf->n_coll >= (1u << 24)) return O2TPC_EINVAL;
    for (uint64_t i = 0; i < tf->n_coll; ++i) {
      const double v = tf->coll_time[i];
      if (!std::isfinite(v) || (i > 0 && v < tf->coll_time[i - 1])) return O2TPC_EINVAL;
    }
  }
  if (tf->n >= kMaxBatchHits) return O2TPC_ETOOBIG;
  if ((c->cfg.flags & O2TPC_FLAG_COMPRESS) && tf->n > kMaxCompressHits) return O2TPC_ETOOBIG;
  if (footprint_of(tf->n, (c->cfg.flags & O2TPC_FLAG_COMPRESS) != 0) > c->cfg.mem_budget) return O2TPC_ETOOBIG;
  return O2TPC_OK;
}

int o2tpc_submit_many(o2tpc_ctx* ctx, const o2tpc_tf* tfs, uint32_t n, uint64_t* tickets) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || (n > 0 && (!tfs || !tickets))) return O2TPC_EINVAL;
  std::vector<std::shared_ptr<Job>> js(n);
  const double t = now_ms();
  for (uint32_t i = 0; i < n; ++i) {
    int rc = check_tf(c, &tfs[i]);
    if (rc != O2TPC_OK) return rc;
    js[i] = std::make_shared<Job>();
    js[i]->tf = tfs[i];
    js[i]->footprint = footprint_of(tfs[i].n, (c->cfg.flags & O2TPC_FLAG_COMPRESS) != 0);
    js[i]->t_submit = t;
  }
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->fatal != O2TPC_OK) return c->fatal;
    if ((uint64_t)c->inflight + n > (uint64_t)c->cfg.max_inflight) return O2TPC_EAGAIN;
    for (uint32_t i = 0; i < n; ++i) {
      js[i]->ticket = c->nextTicket++;
      c->jobs[js[i]->ticket] = js[i];
      c->queue.push_back(js[i]);
      ++c->inflight;
      tickets[i] = js[i]->ticket;
    }
  }
  c->cvWork.notify_one();
  c->cvUp.notify_all();
  return O2TPC_OK;
}

int o2tpc_submit_tf(o2tpc_ctx* ctx, const o2tpc_tf* tf, uint64_t* ticket) {
  if (!ctx || !tf || !ticket) return O2TPC_EINVAL;
  return o2tpc_submit_many(ctx, tf, 1, ticket);
}

int o2tpc_get_tuning(o2tpc_ctx* ctx, o2tpc_tuning* out) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !out) return O2TPC_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->tune;
  return O2TPC_OK;
}

int o2tpc_poll(o2tpc_ctx* ctx, uint64_t ticket, int32_t timeout_ms, const o2tpc_result** out) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !out) return O2TPC_EINVAL;
  std::unique_lock<std::mutex> lk(c->mu);
  auto it = c->jobs.find(ticket);
  if (it == c->jobs.end()) return O2TPC_ENOTFOUND;
  std::shared_ptr<Job> j = it->second;
  auto ready = [&] { return j->done; };
  if (timeout_ms < 0) c->cvDone.wait(lk, ready);
  else if (!c->cvDone.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return O2TPC_PENDING;
  *out = &j->res;
  return O2TPC_OK;
}

void o2tpc_result_release(o2tpc_ctx* ctx, const o2tpc_result* res) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !res) return;
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto it = c->jobs.begin(); it != c->jobs.end(); ++it) {
      if (&it->second->res == res && it->second->done) {
        j = it->second;
        c->jobs.erase(it);
        --c->inflight;
        break;
      }
    }
  }
  // dropping j releases its results and its reference on the kept stages
  if (j) {
    c->pinned_put(j->host, j->hostBytes);
    j->host = nullptr;
    if (j->mem) {
      cudaSetDevice(c->cfg.device);
      j->mem.reset();
    }
  }
}

int o2tpc_destroy(o2tpc_ctx* ctx) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return O2TPC_EINVAL;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->stop = true;
  }
  c->cvWork.notify_all();
  c->cvUp.notify_all();
  if (c->worker.joinable()) c->worker.join();
  if (c->uploader.joinable()) c->uploader.join();
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->finStop = true;
  }
  c->cvFin.notify_all();
  if (c->finisher.joinable()) c->finisher.join();
  int rc = c->fatal;
  cudaSetDevice(c->cfg.device);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& kv : c->jobs) {
      release_upload(c, *kv.second);
      kv.second->mem.reset();
      if (kv.second->host) cudaFreeHost(kv.second->host);
    }
    c->jobs.clear();
  }
  for (auto& kv : c->pinnedFree) cudaFreeHost(kv.second);
  c->pinnedFree.clear();
  c->dev_free(c->dGeom);
  c->dev_free(c->dCounts);
  for (auto& e : c->graphExec)
    if (e) cudaGraphExecDestroy(e);
  if (c->graphMem) c->dev_free(c->graphMem);
  cudaStreamSynchronize(c->stream);
  for (auto& e : c->graphDl)
    if (e) cudaEventDestroy(e);
  if (c->hStage) cudaFreeHost(c->hStage);
  for (auto& e : c->evs)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->evTl)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->evCtf)
    if (e) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->evWait) cudaEventDestroy(c->evWait);
  if (c->evRef) cudaEventDestroy(c->evRef);
  if (c->upStream) {
    cudaStreamSynchronize(c->upStream);
    cudaStreamDestroy(c->upStream);
  }
  if (c->dlStream) {
    cudaStreamSynchronize(c->dlStream);
    cudaStreamDestroy(c->dlStream);
  }
  if (c->ownStream) cudaStreamDestroy(c->stream);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
  return rc;
}

}  // extern "C"

namespace {

template <typename T>
std::vector<T> d2h(const T* d, size_t count) {
  std::vector<T> v(count);
  if (count) CK(cudaMemcpy(v.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost));
  return v;
}

// Builds the named stage array of TF i of a kept batch (TF-local indices).
bool build_stage(const BatchMem& M, int i, const std::string& name, std::vector<char>& out) {
  const int hb = M.tfHitBase[i], he = M.tfHitEnd[i], nh = he - hb;
  const int tlb = M.tfTlBegin[i], tle = M.tfTlBegin[i + 1], ntl = tle - tlb;
  const int stb = M.tfStBegin[i], ste = M.tfStBegin[i + 1], nst = ste - stb;
  auto put = [&](const void* p, size_t bytes) {
    out.resize(bytes);
    if (bytes) memcpy(out.data(), p, bytes);
  };
  auto rel = [](std::vector<int>& v, int base) {
    for (auto& x : v)
      if (x >= 0) x -= base;
  };
  if (name == "sorted_orig") {
    auto v = d2h(M.sorig + hb, nh);
    for (auto& x : v) x -= M.tfInBase[i];
    put(v.data(), v.size() * 4);
  } else if (name == "sorted_yz") {
    auto v = d2h(M.syz + hb, nh);
    put(v.data(), v.size() * 8);
  } else if (name == "row_grid" || name == "cell_start") {
    auto g = d2h(M.grid + (size_t)i * kRowsPerTF, kRowsPerTF);
    const int cb = g[0].cellBase;
    const int ce = g[kRowsPerTF - 1].cellBase + g[kRowsPerTF - 1].ny * g[kRowsPerTF - 1].nz;
    if (name == "row_grid") {
      std::vector<int> v(kRowsPerTF * 8);
      for (int r = 0; r < kRowsPerTF; ++r) {
        v[8 * r + 0] = g[r].start - hb;
        v[8 * r + 1] = g[r].count;
        v[8 * r + 2] = g[r].cellBase - cb;
        v[8 * r + 3] = g[r].ny;
        v[8 * r + 4] = g[r].nz;
        v[8 * r + 5] = g[r].cz;
        v[8 * r + 6] = g[r].zmin;
        v[8 * r + 7] = 0;
      }
      put(v.data(), v.size() * 4);
    } else {
      auto v = d2h(M.cellStart + cb, (size_t)(ce - cb) + 1);
      for (auto& x : v) x -= hb;
      put(v.data(), v.size() * 4);
    }
  } else if (name == "up_raw" || name == "dn_raw" || name == "up" || name == "dn") {
    const int* src = name == "up_raw" ? M.upRaw : name == "dn_raw" ? M.dnRaw : name == "up" ? M.up : M.dn;
    auto v = d2h(src + hb, nh);
    rel(v, hb);
    put(v.data(), v.size() * 4);
  } else if (name == "starts") {
    auto v = d2h(M.starts + tlb, ntl);
    rel(v, hb);
    put(v.data(), v.size() * 4);
  } else if (name == "tl_nhits") {
    auto v = d2h(M.tb.nhits + tlb, ntl);
    put(v.data(), v.size() * 4);
  } else if (name == "tl_hits") {
    auto nhv = d2h(M.tb.nhits + tlb, ntl);
    auto nav = d2h(M.tb.nasc + tlb, ntl);
    auto hv = d2h(M.tb.hits + (size_t)tlb * kMaxTlHits, (size_t)ntl * kMaxTlHits);
    std::vector<int> v((size_t)ntl * kMaxTlHits, -1);
    for (int k = 0; k < ntl; ++k) {
      const int nhk = nhv[k], na = nav[k], nd = nhk - na;
      int m = 0;
      for (int j = 0; j < nhk; ++j) {
        const int q = (j < nd) ? (nhk - 1 - j) : (j - nd);
        v[(size_t)k * kMaxTlHits + m++] = hv[(size_t)k * kMaxTlHits + q] - hb;
      }
    }
    put(v.data(), v.size() * 4);
  } else if (name == "tl_state") {
    auto v = d2h(M.tb.state + (size_t)tlb * 21, (size_t)ntl * 21);
    put(v.data(), v.size() * 4);
  } else if (name == "st_tracklet") {
    auto v = d2h(M.sb.tl + stb, nst);
    rel(v, tlb);
    put(v.data(), v.size() * 4);
  } else if (name == "st_off" || name == "st_hits") {
    auto off = d2h(M.sb.off + stb, (size_t)nst + 1);
    if (name == "st_off") {
      const int o0 = off[0];
      for (auto& x : off) x -= o0;
      put(off.data(), off.size() * 4);
    } else {
      auto v = d2h(M.sb.hits + off[0], (size_t)(off[nst] - off[0]));
      rel(v, hb);
      put(v.data(), v.size() * 4);
    }
  } else if (name == "st_in" || name == "st_out") {
    auto v = d2h((name == "st_in" ? M.sb.in : M.sb.out) + (size_t)stb * 21, (size_t)nst * 21);
    put(v.data(), v.size() * 4);
  } else if (name == "st_next" || name == "st_prev") {
    auto v = d2h((name == "st_next" ? M.mb.next : M.mb.prev) + stb, nst);
    rel(v, stb);
    put(v.data(), v.size() * 4);
  } else {
    return false;
  }
  return true;
}

}  // namespace

extern "C" int o2tpc_get_stage(o2tpc_ctx* ctx, uint64_t ticket, const char* name, void* dst, uint64_t capacity,
                               uint64_t* needed) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !name) return O2TPC_EINVAL;
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->jobs.find(ticket);
    if (it == c->jobs.end() || !it->second->done) return O2TPC_ENOTFOUND;
    j = it->second;
  }
  if (!j->mem) return O2TPC_EINVAL;
  std::vector<char> buf;
  try {
    cudaSetDevice(c->cfg.device);
    if (!build_stage(*j->mem, j->tfIndex, name, buf)) return O2TPC_EINVAL;
  } catch (const CudaError&) {
    cudaGetLastError();
    return O2TPC_ECUDA;
  }
  if (needed) *needed = buf.size();
  if (!dst || capacity < buf.size()) return O2TPC_EINVAL;
  if (!buf.empty()) memcpy(dst, buf.data(), buf.size());
  return O2TPC_OK;
}
