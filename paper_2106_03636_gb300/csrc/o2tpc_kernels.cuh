// o2tpc_kernels.cuh - launchers of the tracker kernels (host side) and the
// device buffers they work on.
#pragma once

#include <climits>

#include "o2tpc_internal.cuh"

namespace o2tpc {

// Kernels launched by the calling host thread (each launcher adds its own).
extern thread_local long long g_launch_count;

constexpr int kNFBlock = 128;      // default hits per NeighboursFinder block
constexpr int kMaxTlHits = kNRow;  // hit slots per tracklet

// k_bin.cu
void launch_ingest_stats(const TFDesc* tfs, const int2* tiles, int nTiles, int tileSize, const GeomConst* G,
                         int* tileStats, unsigned* err, cudaStream_t st);
void launch_row_reduce(const TFDesc* tfs, int nTF, int* tileStats, int* rowCnt, int* rowMin, int* rowMax,
                       cudaStream_t st);
void launch_grid(int nRows, const int* rowCnt, const int* rowMin, const int* rowMax, const GeomConst* G,
                 RowGrid* grid, int* nfBlockStart, int nfBlock, int* totals, cudaStream_t st);
void launch_row_scatter(const TFDesc* tfs, const int2* tiles, int nTiles, int tileSize, const GeomConst* G,
                        const int* tileStats, const RowGrid* grid, int4* bucket, cudaStream_t st);
void launch_cell_sort(int nRows, const RowGrid* grid, const int4* bucket, int* cellStart, int2* syz, int* sorig,
                      int* gscratch, const int* totals, cudaStream_t st,
                      int threadsPerRow = 256);

// k_ca.cu
// syz must hold one int2 of padding past the last hit (the 16-byte aligned
// slab copies may read it); err collects kErrTimeout.  inject: the context's
// debug_inject bits (bit 0: staged slabs armed but not copied, short waits).
void launch_neighbours(int nfBlocks, int hitsPerBlock, bool stage, const RowGrid* grid, const int* nfBlockStart,
                       int nRows, const int* cellStart, const int2* syz, const GeomConst* G, int* upRaw, int* dnRaw,
                       unsigned* err, cudaStream_t st, unsigned inject = 0);
// Row step 2: links across one missing row for the hits that found no
// adjacent-row pair (after launch_neighbours; n sizes the grid).
void launch_neighbours_gap(int n, const int* nDev, const RowGrid* grid, int nRows, const int* cellStart,
                           const int2* syz, const GeomConst* G, int* upRaw, int* dnRaw, cudaStream_t st);
// Data-dependent sizes are read by the kernels from device memory (nDev,
// the fields of Counts); the host-side n of a launcher only sizes its grid:
// the exact size on the regular path, a capacity on the captured path.
struct Counts {
  int n;         // clusters of the batch
  int nTl;       // start hits = tracklets
  int nSt;       // sector tracks
  int nStHits;   // their hits
  int nHeads;    // merged tracks
  int overflow;  // a capacity was exceeded (captured path: rerun on the regular path)
  int nKeys;     // merge lists / directed sector edges of the batch
  int pad;
};
void launch_clean(int n, const int* nDev, const int* upRaw, const int* dnRaw, int* up, int* dn, int* startFlag,
                  cudaStream_t st);
int scan_scratch_ints(long long n);
void scan_exclusive(const int* in, int* out, int n, const int* nDev, int* scratch, cudaStream_t st);
// perm[0, m) = 0..m-1 (m = *nDev <= n) ordered by descending length
// off[i + 1] - off[i] (lengths clamped to kLenBins - 1; any order among equal
// lengths), so that a kernel walking perm with one thread per item gives the
// 32 lanes of a warp items of about equal length.  hist: kLenBins ints.
constexpr int kLenBins = 512;
void launch_len_order(int n, const int* nDev, const int* off, int* hist, int* perm, cudaStream_t st);
// Ordered compaction with warp ballots: the indices i < *nDev with flag[i]
// set, ascending, into out (at most cap; more raise *overflow).
// launch_ballot_count: tile counts, their scan into tileOff and *count;
// launch_ballot_compact: the writes.  tileCnt/tileOff: ballot_tiles(n) + 1.
int ballot_tiles(long long n);
void launch_ballot_count(int n, const int* nDev, const int* flag, int* tileCnt, int* tileOff, int* count, int cap,
                         int* overflow, int* scratch, cudaStream_t st);
void launch_ballot_compact(int n, const int* nDev, const int* flag, const int* tileOff, int* out, int cap,
                           int* overflow, cudaStream_t st);
// *dst = min(arr[*idx], cap); optionally *dst2 = min(arr2[*idx], cap2) and
// endBase[*dst] = *dst2
void launch_count_at(const int* arr, const int* idx, int* dst, int cap, int* overflow, cudaStream_t st,
                     const int* arr2 = nullptr, int* dst2 = nullptr, int cap2 = 0, int* endBase = nullptr);
void launch_iota(int* out, int n, cudaStream_t st);  // out[i] = i
// An empty kernel: ends a stream's work of a batch on the compute engine, so
// that the stream's next operations do not queue behind copies of other
// streams on the copy engine that served its last copy.
void launch_stream_tail(cudaStream_t st);
void launch_tf_ranges(int nTF, const RowGrid* grid, const int* list, const int* nListDev, int* tfBegin,
                      cudaStream_t st);
void launch_lower_bounds(const int* list, const int* nListDev, const int* keys, int nKeys, int* out,
                         cudaStream_t st);

// k_track.cu
struct TrackletBufs {
  int* nhits;    // [nTl]  total attached hits (0: dropped)
  int* nasc;     // [nTl]  hits in slots [0, nasc) in ascending rows; slots [nasc, nhits) descending
  int* hits;     // [nTl * kMaxTlHits]
  uint8_t* rows; // [nTl * kMaxTlHits]
  float* state;  // [nTl * 21]  x, par[5], cov[15] at the innermost hit
  int* zref;     // [nTl]
  int* yref;     // [nTl]  y origin (units) of the state handed between the passes
  int* rbase;    // [nTl]  batch-global row of pad row 0 of the tracklet's sector
};
// passEnd: optional 4 events recorded after the chain-fit, outward, refit and
// inward passes.  coopSearch: the following passes scan the row windows
// cooperatively over the warp instead of lane by lane (identical results).
// nTl sizes the grids; the kernels read the count at nTlDev
void launch_tracklets(int nTl, const int* nTlDev, int* workCounter, const int* starts, const int* up,
                      const RowGrid* grid, int nRows, const int* cellStart, const int2* syz, const GeomConst* G,
                      TrackletBufs tb, cudaStream_t st, cudaEvent_t* passEnd = nullptr, bool coopSearch = false);

struct SectorTrackBufs {
  int* tl;        // [nSt] tracklet of the sector track
  int* sector;    // [nSt] sector 0..35
  int* tf;        // [nSt] TF index in the batch
  int* zref;      // [nSt]
  int* off;       // [nSt + 1] into hits
  int* hits;      // sorted hit indices, ascending rows
  uint8_t* rows;  // row of each hit
  int2* yz;       // coordinates of each hit (gathered once for the fits)
  int* orig;      // batch-global input index of each hit
  float* in;      // [nSt * 21] state at the innermost hit (inward fit)
  float* out;     // [nSt * 21] state at the outermost hit (outward fit)
};
// Ownership over w (n words: 32-bit keys, or 64-bit when *wide is set by the
// sector ranges; w must hold 8 bytes per hit and start at zero).
void launch_ownership(int nTl, const int* nTlDev, int nSec, const RowGrid* grid, const int* starts, TrackletBufs tb,
                      void* w, int* secBegin, int* wide, cudaStream_t st);
void launch_segments_count(int nTl, const int* nTlDev, const int* secBegin, const int* wide, const void* w,
                           TrackletBufs tb, int* nSeg, int* nSegHits, cudaStream_t st);
// capSt / capHits: room in the sector-track buffers (writes past them dropped)
void launch_segments_write(int nTl, const int* nTlDev, const int* secBegin, const int* wide, const void* w,
                           TrackletBufs tb, const int* segPos, const int* segHitPos, const int2* syz,
                           const int* sorig, SectorTrackBufs sb, int capSt, int capHits, cudaStream_t st);
// sb.yz / sb.orig of every sector-track hit (after the CSR end is written)
void launch_st_gather(int nHits, const int* nHitsDev, SectorTrackBufs sb, const int2* syz, const int* sorig,
                      cudaStream_t st);
// order: the sector tracks in the order the fits take them (launch_len_order of sb.off)
void launch_sector_fit(int nSt, const int* nStDev, const TrackletBufs tb, const int2* syz, const GeomConst* G,
                       SectorTrackBufs sb, const int* order, cudaStream_t st);

// k_merge.cu
struct MergeBufs {
  int* keyIn;        // [nSt] B-list key of the inner end (-1: not a border end)
  int* keyOut;       // [nSt] edge key of the outer end (-1)
  int* listCnt;      // [nKeys + 1]
  int* listStart;    // [nKeys + 1]
  int* listItems;    // [nSt]
  int* listKey;      // [nSt] drift coordinate (units) of each list item
  float4* pairs;     // [cap] {chi2, a, b, edge}
  int* pairCount;    // [1]
  int pairCap;
  float4* pairsSorted;  // [cap]
  float4* sortScratch;  // [2 * max(cap, nSt)] padded bitonic buffers of the lists (int2);
                        // then the per-track minima of the pair selection (2 * nSt u64)
  int nSt;
  int* edgeCnt;      // [nKeys + 1]
  int* edgeStart;    // [nKeys + 1]
  int* next;         // [nSt]
  int* prev;         // [nSt]
  int* reached;      // [nSt]
  const Counts* cnt; // device sizes (nSt, nKeys)
};
constexpr int kMaxChain = 64;  // segments per merged chain, at most
void launch_merge_keys(int nSt, const SectorTrackBufs sb, const GeomConst* G, MergeBufs mb, int nKeys, int* scratch,
                       cudaStream_t st);
void launch_merge_pairs(int nSt, const SectorTrackBufs sb, const GeomConst* G, MergeBufs mb, unsigned* err,
                        cudaStream_t st);
void launch_merge_select(int nPairs, int nKeys, MergeBufs mb, int* scratch, cudaStream_t st);
void launch_chains(int nSt, MergeBufs mb, int* headFlag, cudaStream_t st);
void launch_chain_counts(int nHeads, const int* nHeadsDev, const int* heads, const SectorTrackBufs sb, MergeBufs mb,
                         int* trkNcl, cudaStream_t st);

struct OutBufs {
  int* off;         // [nTrk + 1] batch-global offsets into cl
  int* cl;          // input index of each cluster inside its TF
  float* x;
  float* alpha;
  float* par;       // [nTrk * 5]
  float* cov;       // [nTrk * 15]
  float* chi2;
  int* ndf;
  uint8_t* sector;
  uint8_t* flags;
  int* zref;
  int* nFallback;   // [1]
  int* fallback;    // [nTrk] tracks queued for the FP64 refit
  // ends of each track, written by the final refit for the continuous-readout
  // stage: {zeta min, zeta max of the two end clusters, zeta of the first
  // cluster, of the last} and
  // {first row | last row << 8 | first sector << 16 | last sector << 24, TF}
  int4* ends;
  int2* endsR;
  // continuous-readout results
  float* t0;        // us
  float* t0err;
  float* t0lo;
  float* t0hi;
  int* mate;        // track linked across the central membrane, or -1
  int* coll;        // interaction time index inside the TF, or -1
};
void launch_final_refit(int nHeads, const int* nHeadsDev, const int* heads, const SectorTrackBufs sb, MergeBufs mb,
                        const int2* syz, const int* sorig, const TFDesc* tfs, const GeomConst* G, int forceFp64,
                        OutBufs ob, cudaStream_t st);
// Compressed TF (csrc/k_ctf.cu).  Stream table entry: first symbol, symbol
// count, first chunk, chunk count.
struct CtfStream {
  long long start, count;
  int chunk0, nChunks;
};
constexpr int kCtfChunkBytes = 6160;  // >= 4 + 1.5 * 4096 + 4: a coded chunk at most (multiple of 16)
struct CtfBufs {
  uint8_t* onTrack;    // [n + 1] input cluster on a track
  int* firstFlag;      // [n + 1] input index of a kept track's first cluster
  int* trkAtFirst;     // [n]
  int* unFlag;         // [n + 1] sorted hit on no track
  int* canonFirst;     // [nTrk] first-cluster input indices of kept tracks, ascending
  int* canonTrk;       // [nTrk] the tracks in that order
  int* len;            // [nTrk + 1] their cluster counts
  int* lenScan;        // [nTrk + 1]
  int* unList;         // [n] sorted hits on no track, ascending
  int* inBase;         // [nTF + 1]
  int* tfKt;           // [nTF + 1] kept-track list range of each TF
  int* tfUn;           // [nTF + 1] free-cluster list range of each TF
  int* counts;         // [4] kept tracks, free clusters, chunks
  int* tfCounts;       // [nTF * 3] header counts
  CtfStream* sd;       // [nTF * 10]
  uint8_t* sym;        // [8 nSeqCap + 2 nTrkCap] byte planes
  long long nSeqCap, nTrkCap;
  int chunkCap;
  unsigned* hist;      // [nTF * 10 * 256]
  uint16_t* freq;      // [nTF * 10 * 256]
  uint2* enc;          // [nTF * 10 * 256] coding entries (start | freq << 16, 1 / freq)
  int* degen;          // [nTF * 10] 1: one symbol holds the whole table (nothing to code)
  uint8_t* scratch;    // [chunkCap * kCtfChunkBytes]
  int* bytes;          // [chunkCap + 1] coded chunk sizes
  int* payOff;         // [chunkCap + 1]
  long long* tfBlob;   // [nTF + 1] blob offset of each TF, total at nTF
  long long* tfHead;   // [nTF] header bytes of each TF
};
int ctf_chunk_cap(long long nSeqCap, long long nTrkCap, int nTF);
// Everything up to the blob sizes (cb.tfBlob); then, with the blob
// allocated, the headers and payload copies.
void launch_ctf_symbols(int n, const int* nDev, int nTrk, const int* nTrkDev, int nTF, const TFDesc* tfs,
                        const RowGrid* grid, int nRows, const int2* syz, const int* sorig, const int* heads,
                        SectorTrackBufs sb, MergeBufs mb, OutBufs ob, CtfBufs cb, int* tileCnt, int* tileOff,
                        int* overflow, int* scratch, cudaStream_t st);
void launch_ctf_blob(int nTF, CtfBufs cb, uint8_t* blob, cudaStream_t st);
// Sorts every list of mb (listStart, listKey, listItems) by key, then item.
void launch_list_sort(int nKeys, MergeBufs mb, cudaStream_t st);
// Continuous-readout stage over the batch's nTrk (capacity) tracks.  mb: the
// merger's buffers, free by then, except next / prev / pairCount, which must
// be the stage's own (nTrk links, one count); pairCap bounds the membrane
// pairs (more set kErrMembrane in err).  coll: the batch's interaction times
// (TFDesc ranges); trkTfBegin: first track of each TF (partners are written
// as indices inside their TF).
void launch_continuous(int nTrk, const int* nTrkDev, int nKeys, OutBufs ob, MergeBufs mb, const GeomConst* G,
                       const TFDesc* tfs, const double* coll, const int* trkTfBegin, unsigned* err, int* scratch,
                       cudaStream_t st);

}  // namespace o2tpc
