// k_bin.cu - ingest, per-row statistics, grid and the stable per-row sort.
//
// Steps A1-A4 of the hot path: clusters of a batch of Time Frames are
// decoded to integer (y, zeta), counted per (TF, sector, row), binned into a
// per-row grid of cells (cell = iz * ny + iy) and sorted by
// (TF, sector, row, cell, input index).  The sort is a two-level counting
// sort: tiles of the input scatter into row buckets at offsets from a
// per-(tile,row) prefix (no global atomics), then one CTA per row scatters
// its bucket into cells and restores input order inside each cell, so the
// result is the stable order whatever the atomic interleaving.
#include "o2tpc_kernels.cuh"

namespace o2tpc {

// Decodes cluster i of TF t.  Returns false (and sets the error word) for
// invalid content; the cluster is then filed under row 0 so that indices stay
// in bounds.
__device__ inline bool decode(const TFDesc& t, int i, const GeomConst* __restrict__ G, int& lr, int& yu,
                              int& zu) {
  int s, r;
  bool ok = true;
  if (t.format == 1) {
    const uint32_t* rec = reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(t.in0) + 12ll * i);
    uint32_t w0 = __ldg(rec), w1 = __ldg(rec + 1), w2 = __ldg(rec + 2);
    uint32_t pad = w1 & 0xFFFFu;
    r = (int)(w2 & 0xFFu);
    s = (int)((w2 >> 8) & 0xFFu);
    if (s >= kNSec || r >= kNRow || w0 > 0x3FFFFFFFu) { ok = false; s = 0; r = 0; }
    yu = (int)pad - 32 * G->npads[r];
    zu = (int)w0;
  } else {
    s = __ldg(static_cast<const uint8_t*>(t.in0) + i);
    r = __ldg(static_cast<const uint8_t*>(t.in1) + i);
    float yf = __ldg(t.y + i), zf = t.z ? __ldg(t.z + i) : __ldg(t.time + i);
    if (s >= kNSec || r >= kNRow) { ok = false; s = 0; r = 0; }
    if (!isfinite(yf) || !isfinite(zf)) { ok = false; yf = 0.f; zf = 0.f; }
    float yq = rintf(__fmul_rn(yf, 160.0f));
    float zq;
    if (t.z) {
      const float d = (s < 18) ? __fsub_rn(250.0f, zf) : __fadd_rn(250.0f, zf);
      zq = rintf(__fmul_rn(d, G->kz));
    } else {
      zq = rintf(__fmul_rn(zf, 320.0f));  // drift time (us) -> 1/64 of a 200 ns bin
    }
    if (fabsf(yq) > 1048576.0f || fabsf(zq) > 1073741824.0f) { ok = false; yq = 0.f; zq = 0.f; }
    yu = (int)yq;
    zu = (int)zq;
  }
  lr = s * kNRow + r;
  return ok;
}

// K0: per tile, decode and accumulate per-row count / min / max in shared
// memory; write the tile's 5472-row statistics (SoA: count, zmin, zmax).
__global__ void __launch_bounds__(512) k_ingest_stats(const TFDesc* __restrict__ tfs, const int2* __restrict__ tiles,
                                                      int tileSize, const GeomConst* __restrict__ G,
                                                      int* __restrict__ tileStats, unsigned* __restrict__ err) {
  extern __shared__ int sm[];
  int* s_cnt = sm;
  int* s_min = sm + kRowsPerTF;
  int* s_max = sm + 2 * kRowsPerTF;
  const int tile = blockIdx.x;
  const int2 td = tiles[tile];
  const TFDesc t = tfs[td.x];
  for (int i = threadIdx.x; i < kRowsPerTF; i += blockDim.x) { s_cnt[i] = 0; s_min[i] = INT_MAX; s_max[i] = INT_MIN; }
  __syncthreads();
  const int b = td.y, e = min(t.n, td.y + tileSize);
  bool bad = false;
  for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
    int lr, yu, zu;
    if (!decode(t, i, G, lr, yu, zu)) bad = true;
    atomicAdd(&s_cnt[lr], 1);
    atomicMin(&s_min[lr], zu);
    atomicMax(&s_max[lr], zu);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrInput);
  int* out = tileStats + (size_t)tile * 3 * kRowsPerTF;
  for (int i = threadIdx.x; i < kRowsPerTF; i += blockDim.x) {
    out[i] = s_cnt[i];
    out[kRowsPerTF + i] = s_min[i];
    out[2 * kRowsPerTF + i] = s_max[i];
  }
}

// Per (TF, row): reduce the tile statistics, and turn each tile's count into
// its exclusive offset inside the row's bucket (tile order = input order).
// A block takes 32 rows of one TF; its 32 warps split the TF's tiles into 32
// consecutive chunks (lane = row, so a warp's loads of one tile are one
// 128-byte line): chunk sums first, their exclusive scan per row in shared
// memory, then each chunk writes its tiles' offsets.
constexpr int kRRRows = 32, kRRChunks = 32;
__global__ void __launch_bounds__(kRRRows * kRRChunks) k_row_reduce(const TFDesc* __restrict__ tfs, int nTF,
                                                                  int* __restrict__ tileStats, int* __restrict__ rowCnt,
                                                                  int* __restrict__ rowMin, int* __restrict__ rowMax) {
  __shared__ int s_sum[kRRChunks][kRRRows + 1], s_min[kRRChunks][kRRRows + 1], s_max[kRRChunks][kRRRows + 1];
  const int blocksPerTF = (kRowsPerTF + kRRRows - 1) / kRRRows;
  const int tf = blockIdx.x / blocksPerTF;
  const int lane = threadIdx.x % kRRRows, q = threadIdx.x / kRRRows;
  const int lr = (blockIdx.x % blocksPerTF) * kRRRows + lane;
  const bool row = tf < nTF && lr < kRowsPerTF;
  const TFDesc t = tfs[min(tf, nTF - 1)];
  const int per = (t.nTiles + kRRChunks - 1) / kRRChunks;
  const int k0 = min(q * per, t.nTiles), k1 = min(k0 + per, t.nTiles);
  int c = 0, mn = INT_MAX, mx = INT_MIN;
  if (row)
    for (int k = k0; k < k1; ++k) {
      const int* ts = tileStats + (size_t)(t.tileBase + k) * 3 * kRowsPerTF;
      c += ts[lr];
      mn = min(mn, ts[kRowsPerTF + lr]);
      mx = max(mx, ts[2 * kRowsPerTF + lr]);
    }
  s_sum[q][lane] = c;
  s_min[q][lane] = mn;
  s_max[q][lane] = mx;
  __syncthreads();
  if (q == 0) {  // per row: exclusive scan of the chunk sums, totals, extremes
    int run = 0, m0 = INT_MAX, m1 = INT_MIN;
    for (int j = 0; j < kRRChunks; ++j) {
      const int v = s_sum[j][lane];
      s_sum[j][lane] = run;
      run += v;
      m0 = min(m0, s_min[j][lane]);
      m1 = max(m1, s_max[j][lane]);
    }
    if (row) {
      const int g = tf * kRowsPerTF + lr;
      rowCnt[g] = run;
      rowMin[g] = m0;
      rowMax[g] = m1;
    }
  }
  __syncthreads();
  if (row) {
    int o = s_sum[q][lane];
    for (int k = k0; k < k1; ++k) {
      int* ts = tileStats + (size_t)(t.tileBase + k) * 3 * kRowsPerTF;
      const int v = ts[lr];
      ts[lr] = o;
      o += v;
    }
  }
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024).
__device__ inline int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  int incl = x + (w > 0 ? ws[w - 1] : 0);
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return incl - v;
}

// Grid of every row and the three row-level exclusive scans (hits, cells,
// NeighboursFinder blocks).  One CTA of 1024 threads; each thread owns a
// contiguous run of rows.  totals[0..2] = hits, cells, NF blocks.
__global__ void __launch_bounds__(1024) k_grid(int nRows, const int* __restrict__ rowCnt, const int* __restrict__ rowMin,
                                               const int* __restrict__ rowMax, const GeomConst* __restrict__ G,
                                               RowGrid* __restrict__ grid, int* __restrict__ nfBlockStart,
                                               int nfBlock, int* __restrict__ totals) {
  int per = (nRows + blockDim.x - 1) / blockDim.x;
  int b = threadIdx.x * per, e = min(nRows, b + per);
  int sh = 0, sc = 0, sb = 0;
  for (int R = b; R < e; ++R) {
    int r = (R % kRowsPerTF) % kNRow;
    int n = rowCnt[R];
    int ny = max(1, (64 * G->npads[r] + kCellY - 1) / kCellY);
    int nz = 1;
    if (n > 0) nz = min(max((n + kHitsPerCell * ny - 1) / (kHitsPerCell * ny), 1), kMaxNz);
    sh += n;
    sc += ny * nz;
    sb += (n + nfBlock - 1) / nfBlock;
  }
  int th, tc, tb;
  int oh = block_excl_scan(sh, &th);
  int oc = block_excl_scan(sc, &tc);
  int ob = block_excl_scan(sb, &tb);
  for (int R = b; R < e; ++R) {
    int r = (R % kRowsPerTF) % kNRow;
    int n = rowCnt[R];
    RowGrid g;
    g.ny = max(1, (64 * G->npads[r] + kCellY - 1) / kCellY);
    g.nz = 1;
    g.cz = 1;
    g.zmin = 0;
    if (n > 0) {
      g.nz = min(max((n + kHitsPerCell * g.ny - 1) / (kHitsPerCell * g.ny), 1), kMaxNz);
      long long range = (long long)rowMax[R] - (long long)rowMin[R] + 1;
      g.cz = (int)((range + g.nz - 1) / g.nz);
      g.zmin = rowMin[R];
    }
    g.start = oh;
    g.count = n;
    g.cellBase = oc;
    g.pad = 0;
    grid[R] = g;
    nfBlockStart[R] = ob;
    oh += n;
    oc += g.ny * g.nz;
    ob += (n + nfBlock - 1) / nfBlock;
  }
  if (threadIdx.x == 0) {
    totals[0] = th;
    totals[1] = tc;
    totals[2] = tb;
    nfBlockStart[nRows] = tb;
  }
}

__global__ void k_cell_sentinel(int* __restrict__ cellStart, const int* __restrict__ totals) {
  cellStart[totals[1]] = totals[0];
}

// K3a: scatter each tile's clusters into its row bucket at
// rowStart + (tile offset within the row) + (unordered rank inside the tile).
// Records: {y_u, zeta_u, batch input index, cell}.  Persistent: one CTA per
// SM takes the tiles in turn, so that only one tile per SM is open at a time
// and the partly written 32-byte sectors of its 5472 row segments stay in L2
// until they fill (with one CTA per tile the whole grid's open sectors
// outgrew L2 on a 128-orbit TF).  Each thread decodes kU clusters before the
// first of their scattered stores, which keeps kU input loads in flight.
#ifndef O2TPC_SCATTER_THREADS
#define O2TPC_SCATTER_THREADS 1024
#endif
#ifndef O2TPC_SCATTER_UNROLL
#define O2TPC_SCATTER_UNROLL 4
#endif
constexpr int kScatterT = O2TPC_SCATTER_THREADS, kScatterU = O2TPC_SCATTER_UNROLL;
__global__ void __launch_bounds__(kScatterT) k_row_scatter(const TFDesc* __restrict__ tfs, const int2* __restrict__ tiles,
                                                           int nTiles, int tileSize, const GeomConst* __restrict__ G,
                                                           const int* __restrict__ tileStats,
                                                           const RowGrid* __restrict__ grid, int4* __restrict__ bucket) {
  __shared__ int s_cur[kRowsPerTF];
  for (int tile = blockIdx.x; tile < nTiles; tile += gridDim.x) {
    const int2 td = tiles[tile];
    const TFDesc t = tfs[td.x];
    const int b = td.y, e = min(t.n, td.y + tileSize);
    if (b >= e) continue;  // an unused tile slot (block-uniform)
    const int Rbase = td.x * kRowsPerTF;
    const int* ts = tileStats + (size_t)tile * 3 * kRowsPerTF;
    __syncthreads();  // the previous tile's slot counters are no longer in use
    for (int i = threadIdx.x; i < kRowsPerTF; i += kScatterT) s_cur[i] = grid[Rbase + i].start + ts[i];
    __syncthreads();
    for (int i0 = b + threadIdx.x; i0 < e; i0 += kScatterT * kScatterU) {
      int lr[kScatterU], yu[kScatterU], zu[kScatterU];
#pragma unroll
      for (int u = 0; u < kScatterU; ++u) {
        const int i = i0 + u * kScatterT;
        if (i < e) decode(t, i, G, lr[u], yu[u], zu[u]);
      }
#pragma unroll
      for (int u = 0; u < kScatterU; ++u) {
        const int i = i0 + u * kScatterT;
        if (i < e) {
          const RowGrid g = grid[Rbase + lr[u]];
          const int iy = cell_iy(g, G->npads[lr[u] % kNRow], yu[u]);
          const int iz = cell_iz_floor(zu[u], g);  // zu >= zmin of its row: 0..nz-1
          const int slot = atomicAdd(&s_cur[lr[u]], 1);
          bucket[slot] = make_int4(yu[u], zu[u], t.inBase + i, iz * g.ny + iy);
        }
      }
    }
  }
}

// K3b: one CTA per row.  Counting sort of the row's bucket by cell into the
// final arrays, then input order restored inside every cell (insertion sort
// by input index).  Cell counters live in shared memory when the row has at
// most kSmemCells cells, else in the global scratch (cellStart itself).
constexpr int kSmemCells = 12288;
constexpr int kRegSort = 8;

template <int kT>
__global__ void __launch_bounds__(kT) k_cell_sort(const RowGrid* __restrict__ grid, const int4* __restrict__ bucket,
                                                   int* __restrict__ cellStart, int2* __restrict__ syz,
                                                   int* __restrict__ sorig, int* __restrict__ gscratch) {
  __shared__ int s_cnt[kSmemCells];
  __shared__ int s_carry;
  const RowGrid g = grid[blockIdx.x];
  if (g.count == 0) {
    for (int c = threadIdx.x; c < g.ny * g.nz; c += blockDim.x) cellStart[g.cellBase + c] = g.start;
    return;
  }
  const int nc = g.ny * g.nz;
  int* cnt = (nc <= kSmemCells) ? s_cnt : (gscratch + g.cellBase);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) cnt[c] = 0;
  __syncthreads();
  const int4* bk = bucket + g.start;
  for (int i = threadIdx.x; i < g.count; i += blockDim.x) atomicAdd(&cnt[bk[i].w], 1);
  __syncthreads();
  // exclusive scan of the cell counts, in chunks of blockDim
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nc; c0 += blockDim.x) {
    int c = c0 + threadIdx.x;
    int v = (c < nc) ? cnt[c] : 0;
    // warp + block scan (up to 1024 threads)
    __shared__ int ws[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int wo = 0;
    for (int k = 0; k < w; ++k) wo += ws[k];
    int excl = s_carry + wo + x - v;
    __syncthreads();
    if (c < nc) {
      cnt[c] = excl;
      cellStart[g.cellBase + c] = g.start + excl;
    }
    if (threadIdx.x == blockDim.x - 1) s_carry = excl + v;
    __syncthreads();
  }
  // scatter (unordered inside a cell)
  for (int i = threadIdx.x; i < g.count; i += blockDim.x) {
    int4 rec = bk[i];
    int pos = g.start + atomicAdd(&cnt[rec.w], 1);
    syz[pos] = make_int2(rec.x, rec.y);
    sorig[pos] = rec.z;
  }
  __syncthreads();
  // restore input order inside each cell: a cell of at most kRegSort hits is
  // loaded at once and sorted in registers (odd-even transposition network);
  // a larger one by insertion in place
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    int b = cellStart[g.cellBase + c];
    int e = (c + 1 < nc) ? cellStart[g.cellBase + c + 1] : g.start + g.count;
    const int m = e - b;
    if (m <= 1) continue;
    if (m <= kRegSort) {
      int ko[kRegSort];
      int2 kv[kRegSort];
#pragma unroll
      for (int j = 0; j < kRegSort; ++j) {
        ko[j] = (j < m) ? sorig[b + j] : INT_MAX;  // input indices are unique and < INT_MAX
        kv[j] = (j < m) ? syz[b + j] : make_int2(0, 0);
      }
#pragma unroll
      for (int rd = 0; rd < kRegSort; ++rd) {
#pragma unroll
        for (int j = rd & 1; j + 1 < kRegSort; j += 2) {
          if (ko[j] > ko[j + 1]) {
            const int tk = ko[j];
            ko[j] = ko[j + 1];
            ko[j + 1] = tk;
            const int2 tv = kv[j];
            kv[j] = kv[j + 1];
            kv[j + 1] = tv;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kRegSort; ++j) {
        if (j < m) {
          sorig[b + j] = ko[j];
          syz[b + j] = kv[j];
        }
      }
      continue;
    }
    for (int i = b + 1; i < e; ++i) {
      int ko = sorig[i];
      int2 kv = syz[i];
      int j = i - 1;
      while (j >= b && sorig[j] > ko) {
        sorig[j + 1] = sorig[j];
        syz[j + 1] = syz[j];
        --j;
      }
      sorig[j + 1] = ko;
      syz[j + 1] = kv;
    }
  }
}

// ------------------------------------------------------------- launchers
void launch_ingest_stats(const TFDesc* tfs, const int2* tiles, int nTiles, int tileSize, const GeomConst* G,
                         int* tileStats, unsigned* err, cudaStream_t st) {
  size_t smem = 3 * kRowsPerTF * sizeof(int);
  cudaFuncSetAttribute(k_ingest_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (nTiles > 0) {
    k_ingest_stats<<<nTiles, 512, smem, st>>>(tfs, tiles, tileSize, G, tileStats, err);
    ++g_launch_count;
  }
}

void launch_row_reduce(const TFDesc* tfs, int nTF, int* tileStats, int* rowCnt, int* rowMin, int* rowMax,
                       cudaStream_t st) {
  if (nTF <= 0) return;
  const int blocksPerTF = (kRowsPerTF + kRRRows - 1) / kRRRows;
  k_row_reduce<<<nTF * blocksPerTF, kRRRows * kRRChunks, 0, st>>>(tfs, nTF, tileStats, rowCnt, rowMin, rowMax);
  ++g_launch_count;
}

void launch_grid(int nRows, const int* rowCnt, const int* rowMin, const int* rowMax, const GeomConst* G,
                 RowGrid* grid, int* nfBlockStart, int nfBlock, int* totals, cudaStream_t st) {
  k_grid<<<1, 1024, 0, st>>>(nRows, rowCnt, rowMin, rowMax, G, grid, nfBlockStart, nfBlock, totals);
  ++g_launch_count;
}

// CTAs per SM of the persistent row scatter
#ifndef O2TPC_SCATTER_CTAS_PER_SM
#define O2TPC_SCATTER_CTAS_PER_SM 1
#endif

void launch_row_scatter(const TFDesc* tfs, const int2* tiles, int nTiles, int tileSize, const GeomConst* G,
                        const int* tileStats, const RowGrid* grid, int4* bucket, cudaStream_t st) {
  if (nTiles > 0) {
    int dev = 0, nSM = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nSM, cudaDevAttrMultiProcessorCount, dev);
    const int nb = nSM > 0 ? std::min(nTiles, nSM * O2TPC_SCATTER_CTAS_PER_SM) : nTiles;
    k_row_scatter<<<nb, kScatterT, 0, st>>>(tfs, tiles, nTiles, tileSize, G, tileStats, grid, bucket);
    ++g_launch_count;
  }
}

void launch_cell_sort(int nRows, const RowGrid* grid, const int4* bucket, int* cellStart, int2* syz, int* sorig,
                      int* gscratch, const int* totals, cudaStream_t st, int threadsPerRow) {
  if (nRows > 0) {
    if (threadsPerRow == 128)
      k_cell_sort<128><<<nRows, 128, 0, st>>>(grid, bucket, cellStart, syz, sorig, gscratch);
    else if (threadsPerRow == 512)
      k_cell_sort<512><<<nRows, 512, 0, st>>>(grid, bucket, cellStart, syz, sorig, gscratch);
    else
      k_cell_sort<256><<<nRows, 256, 0, st>>>(grid, bucket, cellStart, syz, sorig, gscratch);
    ++g_launch_count;
  }
  k_cell_sentinel<<<1, 1, 0, st>>>(cellStart, totals);
  ++g_launch_count;
}

}  // namespace o2tpc
