// o2tpc_static.cu - grid binning and stable sort of one Time Frame without
// any allocation.
//
// Some callers cannot allocate device memory while they run: code inside a
// framework that owns all device memory and hands out only the buffers it
// planned (an inference or reconstruction server with a fixed memory plan),
// code running where a cudaMalloc would synchronise the device or fail
// (inside stream-ordered pipelines, under memory quotas), or embedded users
// that must not grow the process's footprint after start-up.
// o2tpc_sort_tf_static serves them: the caller passes the input clusters and
// the output buffers, and the step's scratch memory (tile statistics, row
// tables, the row-bucket records and the cell counters) lives in file-scope
// device arrays of fixed size, so the call allocates nothing.
//
// The arrays are static __device__ storage: every GPU that loads the library
// holds them (about 6 MB) until the process exits.  Their device addresses
// are looked up once per device with cudaGetSymbolAddress, during the first
// call on that device; that first call should therefore come before any
// stream capture.  Under lazy module loading that first call can also load
// the module and reserve the static storage, so callers with a fixed memory
// plan make one call with n = 0 at start-up.  The cached addresses are not
// valid across a cudaDeviceReset.  All calls share the arrays and leave the
// last call's contents in them, so calls that overlap on the GPU (different
// streams or threads at the same time) race: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "o2tpc.h"
#include "o2tpc_kernels.cuh"

namespace o2tpc {
namespace {

constexpr int kStaticTile = 65536;
constexpr int kStaticTiles = (O2TPC_STATIC_MAX_CLUSTERS + kStaticTile - 1) / kStaticTile;
constexpr long long kStaticCells = O2TPC_STATIC_MAX_CLUSTERS / kHitsPerCell + 46ll * kRowsPerTF + 1;

static __device__ __align__(256) GeomConst s_geom;
static __device__ __align__(256) TFDesc s_tf[1];
static __device__ __align__(256) int2 s_tiles[kStaticTiles];
static __device__ __align__(256) int s_tileStats[kStaticTiles * 3 * kRowsPerTF];
static __device__ __align__(256) int s_rowCnt[kRowsPerTF];
static __device__ __align__(256) int s_rowMin[kRowsPerTF];
static __device__ __align__(256) int s_rowMax[kRowsPerTF];
static __device__ __align__(256) int s_nfBlockStart[kRowsPerTF + 1];
static __device__ __align__(256) int s_totals[4];
static __device__ __align__(256) unsigned s_err[4];
static __device__ __align__(256) int4 s_bucket[O2TPC_STATIC_MAX_CLUSTERS];
static __device__ __align__(256) int s_cellScratch[kStaticCells];

struct StaticPtrs {
  GeomConst* geom;
  TFDesc* tf;
  int2* tiles;
  int* tileStats;
  int *rowCnt, *rowMin, *rowMax, *nfBlockStart, *totals;
  unsigned* err;
  int4* bucket;
  int* cellScratch;
};

std::mutex g_mu;
StaticPtrs g_ptrs[64];
bool g_ready[64];

template <typename T, typename S>
cudaError_t sym(T*& out, const S& symbol) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, symbol);
  out = static_cast<T*>(p);
  return e;
}

// Looks the scratch addresses up once per device (the device must be current).
cudaError_t setup(int dev, StaticPtrs& P) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_ready[dev]) {
    StaticPtrs q{};
    cudaError_t e;
    if ((e = sym(q.geom, s_geom)) != cudaSuccess) return e;
    if ((e = sym(q.tf, s_tf)) != cudaSuccess) return e;
    if ((e = sym(q.tiles, s_tiles)) != cudaSuccess) return e;
    if ((e = sym(q.tileStats, s_tileStats)) != cudaSuccess) return e;
    if ((e = sym(q.rowCnt, s_rowCnt)) != cudaSuccess) return e;
    if ((e = sym(q.rowMin, s_rowMin)) != cudaSuccess) return e;
    if ((e = sym(q.rowMax, s_rowMax)) != cudaSuccess) return e;
    if ((e = sym(q.nfBlockStart, s_nfBlockStart)) != cudaSuccess) return e;
    if ((e = sym(q.totals, s_totals)) != cudaSuccess) return e;
    if ((e = sym(q.err, s_err)) != cudaSuccess) return e;
    if ((e = sym(q.bucket, s_bucket)) != cudaSuccess) return e;
    if ((e = sym(q.cellScratch, s_cellScratch)) != cudaSuccess) return e;
    g_ptrs[dev] = q;
    g_ready[dev] = true;
  }
  P = g_ptrs[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace o2tpc

using namespace o2tpc;

extern "C" int o2tpc_sort_tf_static(const o2tpc_tf* tf, double vdrift_cm_us, int32_t* sorted_orig,
                                    int32_t* sorted_yz, int32_t* row_grid, int32_t* cell_start,
                                    uint64_t cell_capacity, void* stream) {
  if (!tf || !(vdrift_cm_us > 0.0)) return O2TPC_EINVAL;
  if (tf->n > O2TPC_STATIC_MAX_CLUSTERS) return O2TPC_ETOOBIG;
  if (tf->location != O2TPC_LOC_DEVICE) return O2TPC_EINVAL;
  if (tf->format != O2TPC_FMT_FLOAT && tf->format != O2TPC_FMT_FIXED) return O2TPC_EINVAL;
  if (!row_grid || !cell_start || (tf->n > 0 && (!sorted_orig || !sorted_yz))) return O2TPC_EINVAL;
  if (tf->n > 0 && tf->format == O2TPC_FMT_FIXED && !tf->packed) return O2TPC_EINVAL;
  if (tf->n > 0 && tf->format == O2TPC_FMT_FLOAT && (!tf->sector || !tf->row || !tf->y || (!tf->z && !tf->time)))
    return O2TPC_EINVAL;
  const long long cellsMax = (long long)tf->n / kHitsPerCell + 46ll * kRowsPerTF + 1;
  if (cell_capacity < (uint64_t)cellsMax + 1) return O2TPC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return O2TPC_ECUDA;
  StaticPtrs P;
  if (setup(dev, P) != cudaSuccess) {
    cudaGetLastError();
    return O2TPC_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (int)tf->n;
  // descriptors (host copies into the static arrays, in stream order)
  GeomConst g;
  fill_geom(g, 0.5, vdrift_cm_us);  // the field plays no part in binning
  TFDesc d{};
  d.format = tf->format;
  d.n = n;
  d.inBase = 0;
  d.in0 = tf->format == O2TPC_FMT_FIXED ? tf->packed : static_cast<const void*>(tf->sector);
  d.in1 = tf->row;
  d.y = tf->y;
  d.z = tf->z;
  d.time = tf->time;
  d.tileBase = 0;
  d.nTiles = (n + kStaticTile - 1) / kStaticTile;
  int2 tiles[kStaticTiles];
  for (int k = 0; k < d.nTiles; ++k) tiles[k] = make_int2(0, k * kStaticTile);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMemcpyAsync(P.geom, &g, sizeof(g), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(P.tf, &d, sizeof(d), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (d.nTiles > 0 &&
       (e = cudaMemcpyAsync(P.tiles, tiles, sizeof(int2) * d.nTiles, cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
      (e = cudaMemsetAsync(P.err, 0, sizeof(unsigned) * 4, st)) != cudaSuccess) {
    cudaGetLastError();
    return O2TPC_ECUDA;
  }
  RowGrid* grid = reinterpret_cast<RowGrid*>(row_grid);
  launch_ingest_stats(P.tf, P.tiles, d.nTiles, kStaticTile, P.geom, P.tileStats, P.err, st);
  launch_row_reduce(P.tf, 1, P.tileStats, P.rowCnt, P.rowMin, P.rowMax, st);
  launch_grid(kRowsPerTF, P.rowCnt, P.rowMin, P.rowMax, P.geom, grid, P.nfBlockStart, kNFBlock, P.totals, st);
  launch_row_scatter(P.tf, P.tiles, d.nTiles, kStaticTile, P.geom, P.tileStats, grid, P.bucket, st);
  launch_cell_sort(kRowsPerTF, grid, P.bucket, cell_start, reinterpret_cast<int2*>(sorted_yz), sorted_orig,
                   P.cellScratch, P.totals, st);
  unsigned herr = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&herr, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return O2TPC_ECUDA;
  }
  return (herr & kErrInput) ? O2TPC_EINVAL : O2TPC_OK;
}
