// o2tpc_graph.cu - the captured path: the whole pipeline of a batch enqueued
// without one host synchronisation, so that it can be captured once into a
// CUDA graph and replayed for every batch of small and medium Time Frames or
// sub-Time-Frame chunks (one graph launch per batch).
//
// The regular path reads four data-dependent sizes back to the host (start
// hits, sector tracks, merge pairs, merged tracks) to allocate its buffers
// exactly.  Here every buffer comes from one arena sized by capacities derived
// from the largest batch the graph serves (clusters and TFs); every kernel
// takes its size from the device-side Counts record, and every write that a
// capacity bounds is guarded and raises Counts::overflow (the batch is then
// run again on the regular path, so results never depend on the capacities).
#include <algorithm>

#include "o2tpc_graph.cuh"

namespace o2tpc {

namespace {
size_t r256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

GraphCaps graph_caps(long long maxClusters, int maxTFs, bool tight) {
  GraphCaps k{};
  k.nCap = (int)std::max<long long>(maxClusters, 1);
  k.BCap = std::max(maxTFs, 1);
  k.tileSize = kGraphTile;
  k.nTilesCap = k.nCap / k.tileSize + k.BCap + 1;
  k.nRows = k.BCap * kRowsPerTF;
  k.cellsCap = (long long)k.nCap / kHitsPerCell + 46ll * k.nRows + 1;
  // tracklets: chains of >= 3 hits are disjoint, so at most n/3 start hits;
  // 1/8 is 3.5x what the densest workloads produce (overflow: regular path)
  k.tlCap = k.nCap / 8 + 1024;
  // sector tracks own >= 10 hits each, disjoint: at most n/10
  k.stCap = k.nCap / 10 + 1024;
  k.stHitsCap = k.nCap;
  k.headCap = k.stCap;
  k.pairCap = 2 * k.stCap;
  if (tight) k.tlCap = k.stCap = k.headCap = k.pairCap = 16;
  k.nKeys = k.BCap * kNSec * 2;
  k.collCap = 4096 * k.BCap;
  return k;
}

// Carves the arena (base may be null: sizes only); returns the bytes used.
size_t graph_carve(GraphArena& A, char* base) {
  const GraphCaps& k = A.caps;
  size_t off = 0;
  auto take = [&](auto*& p, size_t count) {
    using T = std::remove_reference_t<decltype(*p)>;
    p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += r256(sizeof(T) * std::max<size_t>(count, 1));
  };
  const size_t n = (size_t)k.nCap;
  take(A.tfs, k.BCap);
  take(A.tiles, k.nTilesCap);
  take(A.err, 4);
  take(A.cnt, 1);
  take(A.input, (size_t)12 * n + 64 * k.BCap);
  take(A.tileStats, (size_t)k.nTilesCap * 3 * kRowsPerTF);
  take(A.rowCnt, k.nRows);
  take(A.rowMin, k.nRows);
  take(A.rowMax, k.nRows);
  take(A.grid, k.nRows + 1);
  take(A.nfBlockStart, k.nRows + 1);
  take(A.totals, 4);
  take(A.cellStart, k.cellsCap + 1);
  take(A.gscratch, k.cellsCap);
  take(A.bucket, n);
  take(A.syz, n + 2);
  take(A.sorig, n);
  take(A.upRaw, n);
  take(A.dnRaw, n);
  take(A.up, n);
  take(A.dn, n);
  take(A.flag, n + 1);
  take(A.tileCnt, ballot_tiles((long long)n) + 1);
  take(A.tileOff, ballot_tiles((long long)n) + 1);
  take(A.scratch, scan_scratch_ints((long long)n + 8) + (k.nRows + 8) * 2 / 4096 + 64);
  take(A.starts, k.tlCap);
  take(A.tlTfBegin, k.BCap + 1);
  take(A.tb.nhits, k.tlCap + 1);
  take(A.tb.nasc, k.tlCap);
  take(A.tb.hits, (size_t)k.tlCap * kMaxTlHits);
  take(A.tb.rows, (size_t)k.tlCap * kMaxTlHits);
  take(A.tb.state, (size_t)k.tlCap * 21);
  take(A.tb.zref, k.tlCap);
  take(A.tb.yref, k.tlCap);
  take(A.tb.rbase, k.tlCap);
  take(A.workCounter, 4);
  take(A.w, n);
  take(A.secBegin, k.BCap * kNSec + 1);
  take(A.wide, 1);
  take(A.nSeg, k.tlCap + 1);
  take(A.nSegHits, k.tlCap + 1);
  take(A.segPos, k.tlCap + 1);
  take(A.segHitPos, k.tlCap + 1);
  take(A.sb.tl, k.stCap);
  take(A.sb.sector, k.stCap);
  take(A.sb.tf, k.stCap);
  take(A.sb.zref, k.stCap);
  take(A.sb.off, k.stCap + 1);
  take(A.sb.hits, k.stHitsCap);
  take(A.sb.rows, k.stHitsCap);
  take(A.sb.yz, k.stHitsCap);
  take(A.sb.orig, k.stHitsCap);
  take(A.sb.in, (size_t)k.stCap * 21);
  take(A.sb.out, (size_t)k.stCap * 21);
  take(A.stTfBegin, k.BCap + 1);
  take(A.tfKeys, k.BCap + 1);
  take(A.mb.keyIn, k.stCap);
  take(A.mb.keyOut, k.stCap);
  take(A.mb.listCnt, k.nKeys + 1);
  take(A.mb.listStart, k.nKeys + 1);
  take(A.mb.listItems, k.stCap);
  take(A.mb.listKey, k.stCap);
  take(A.mb.pairCount, 1);
  take(A.mb.edgeCnt, k.nKeys + 1);
  take(A.mb.edgeStart, k.nKeys + 1);
  take(A.mb.next, k.stCap);
  take(A.mb.prev, k.stCap);
  take(A.mb.reached, k.stCap);
  take(A.mb.pairs, k.pairCap);
  take(A.mb.pairsSorted, k.pairCap);
  take(A.mb.sortScratch, 2 * (size_t)std::max(k.pairCap, k.stCap) + 16);
  take(A.headFlag, k.stCap + 1);
  take(A.heads, k.headCap);
  take(A.trkNcl, k.headCap + 1);
  for (OutBufs* o : {&A.ob, &A.ob2}) {
    take(o->off, k.headCap + 1);
    take(o->cl, k.stHitsCap);
    take(o->x, k.headCap);
    take(o->alpha, k.headCap);
    take(o->par, (size_t)k.headCap * 5);
    take(o->cov, (size_t)k.headCap * 15);
    take(o->chi2, k.headCap);
    take(o->ndf, k.headCap);
    take(o->sector, k.headCap);
    take(o->flags, k.headCap);
    take(o->zref, k.headCap);
    take(o->nFallback, 1);
    take(o->fallback, k.headCap);
    take(o->ends, k.headCap);
    take(o->endsR, k.headCap);
    take(o->t0, k.headCap);
    take(o->t0err, k.headCap);
    take(o->t0lo, k.headCap);
    take(o->t0hi, k.headCap);
    take(o->mate, k.headCap);
    take(o->coll, k.headCap);
  }
  take(A.trkTfBegin, k.BCap + 1);
  take(A.lenHist, kLenBins);
  take(A.stOrder, k.stCap);
  take(A.coll, k.collCap);
  take(A.memNext, k.headCap);
  take(A.memPrev, k.headCap);
  take(A.memPairs, 1);
  A.mb.nSt = k.stCap;
  A.mb.pairCap = k.pairCap;
  A.mb.cnt = A.cnt;
  return off;
}

// The batch pipeline with capacities for sizes and no host synchronisation;
// the TF table, tiles and Counts (n, nKeys) are filled before each replay.
void graph_enqueue(const GraphArena& A, const GeomConst* G, int nfBlock, bool nfStage, int sortThreads,
                   int forceFp64, cudaStream_t st, bool coopSearch, bool rowStep2) {
  const GraphCaps& k = A.caps;
  Counts* C = A.cnt;
  const int n = k.nCap;
  cudaMemsetAsync(A.err, 0, 16, st);
  cudaMemsetAsync(&C->nTl, 0, sizeof(int) * 5, st);  // nTl .. overflow
  // A1-A4
  launch_ingest_stats(A.tfs, A.tiles, k.nTilesCap, k.tileSize, G, A.tileStats, A.err, st);
  launch_row_reduce(A.tfs, k.BCap, A.tileStats, A.rowCnt, A.rowMin, A.rowMax, st);
  launch_grid(k.nRows, A.rowCnt, A.rowMin, A.rowMax, G, A.grid, A.nfBlockStart, nfBlock, A.totals, st);
  launch_row_scatter(A.tfs, A.tiles, k.nTilesCap, k.tileSize, G, A.tileStats, A.grid, A.bucket, st);
  launch_cell_sort(k.nRows, A.grid, A.bucket, A.cellStart, A.syz, A.sorig, A.gscratch, A.totals, st, sortThreads);
  // A5-A7
  launch_neighbours(n / nfBlock + k.nRows + 1, nfBlock, nfStage, A.grid, A.nfBlockStart, k.nRows, A.cellStart, A.syz, G,
                    A.upRaw, A.dnRaw, A.err, st);
  if (rowStep2) launch_neighbours_gap(n, &C->n, A.grid, k.nRows, A.cellStart, A.syz, G, A.upRaw, A.dnRaw, st);
  launch_clean(n, &C->n, A.upRaw, A.dnRaw, A.up, A.dn, A.flag, st);
  launch_ballot_count(n, &C->n, A.flag, A.tileCnt, A.tileOff, &C->nTl, k.tlCap, &C->overflow, A.scratch, st);
  launch_ballot_compact(n, &C->n, A.flag, A.tileOff, A.starts, k.tlCap, &C->overflow, st);
  launch_tf_ranges(k.BCap, A.grid, A.starts, &C->nTl, A.tlTfBegin, st);
  // A8
  launch_tracklets(k.tlCap, &C->nTl, A.workCounter, A.starts, A.up, A.grid, k.nRows, A.cellStart, A.syz, G, A.tb,
                   st, nullptr, coopSearch);
  // A9
  cudaMemsetAsync(A.w, 0, sizeof(unsigned long long) * (size_t)n, st);
  launch_ownership(k.tlCap, &C->nTl, k.BCap * kNSec, A.grid, A.starts, A.tb, A.w, A.secBegin, A.wide, st);
  launch_segments_count(k.tlCap, &C->nTl, A.secBegin, A.wide, A.w, A.tb, A.nSeg, A.nSegHits, st);
  scan_exclusive(A.nSeg, A.segPos, k.tlCap, &C->nTl, A.scratch, st);
  scan_exclusive(A.nSegHits, A.segHitPos, k.tlCap, &C->nTl, A.scratch, st);
  launch_segments_write(k.tlCap, &C->nTl, A.secBegin, A.wide, A.w, A.tb, A.segPos, A.segHitPos, A.syz, A.sorig,
                        A.sb, k.stCap, k.stHitsCap, st);
  launch_count_at(A.segPos, &C->nTl, &C->nSt, k.stCap, &C->overflow, st, A.segHitPos, &C->nStHits, k.stHitsCap,
                  A.sb.off);
  launch_st_gather(k.stHitsCap, &C->nStHits, A.sb, A.syz, A.sorig, st);
  launch_len_order(k.stCap, &C->nSt, A.sb.off, A.lenHist, A.stOrder, st);
  launch_sector_fit(k.stCap, &C->nSt, A.tb, A.syz, G, A.sb, A.stOrder, st);
  launch_iota(A.tfKeys, k.BCap + 1, st);
  launch_lower_bounds(A.sb.tf, &C->nSt, A.tfKeys, k.BCap + 1, A.stTfBegin, st);
  // A10
  launch_merge_keys(k.stCap, A.sb, G, A.mb, k.nKeys, A.scratch, st);
  launch_merge_pairs(k.stCap, A.sb, G, A.mb, A.err, st);
  launch_merge_select(k.pairCap, k.nKeys, A.mb, A.scratch, st);
  launch_chains(k.stCap, A.mb, A.headFlag, st);
  launch_ballot_count(k.stCap, &C->nSt, A.headFlag, A.tileCnt, A.tileOff, &C->nHeads, k.headCap, &C->overflow,
                      A.scratch, st);
  launch_ballot_compact(k.stCap, &C->nSt, A.headFlag, A.tileOff, A.heads, k.headCap, &C->overflow, st);
  // A11
  cudaMemsetAsync(A.ob.nFallback, 0, sizeof(int), st);
  launch_chain_counts(k.headCap, &C->nHeads, A.heads, A.sb, A.mb, A.trkNcl, st);
  scan_exclusive(A.trkNcl, A.ob.off, k.headCap, &C->nHeads, A.scratch, st);
  launch_final_refit(k.headCap, &C->nHeads, A.heads, A.sb, A.mb, A.syz, A.sorig, A.tfs, G, forceFp64, A.ob, st);
  launch_lower_bounds(A.heads, &C->nHeads, A.stTfBegin, k.BCap + 1, A.trkTfBegin, st);
  // continuous readout
  MergeBufs mm = A.mb;
  mm.next = A.memNext;
  mm.prev = A.memPrev;
  mm.pairCount = A.memPairs;
  launch_continuous(k.headCap, &C->nHeads, k.nKeys, A.ob, mm, G, A.tfs, A.coll, A.trkTfBegin, A.err, A.scratch, st);
}

}  // namespace o2tpc
