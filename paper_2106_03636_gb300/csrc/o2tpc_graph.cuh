// o2tpc_graph.cuh - arena and launch sequence of the captured path.
#pragma once

#include "o2tpc_kernels.cuh"

namespace o2tpc {

constexpr int kGraphTile = 65536;  // clusters per ingest tile on the captured path

// Capacities of a captured-path arena (from the largest batch it serves).
struct GraphCaps {
  int nCap, BCap, tileSize, nTilesCap, nRows;
  long long cellsCap;
  int tlCap, stCap, stHitsCap, headCap, pairCap, nKeys;
  int collCap;  // interaction times per batch
};

// Every buffer of a batch, carved from one allocation.
struct GraphArena {
  GraphCaps caps{};
  TFDesc* tfs;
  int2* tiles;
  unsigned* err;
  Counts* cnt;
  uint8_t* input;  // host-resident inputs copied here before a replay
  int* tileStats;
  int *rowCnt, *rowMin, *rowMax;
  RowGrid* grid;
  int* nfBlockStart;
  int* totals;
  int* cellStart;
  int* gscratch;
  int4* bucket;
  int2* syz;
  int* sorig;
  int *upRaw, *dnRaw, *up, *dn, *flag, *tileCnt, *tileOff, *scratch;
  int* starts;
  int* tlTfBegin;
  TrackletBufs tb;
  int* workCounter;
  unsigned long long* w;
  int *secBegin, *wide, *nSeg, *nSegHits, *segPos, *segHitPos;
  SectorTrackBufs sb;
  int *stTfBegin, *tfKeys;
  MergeBufs mb;
  int *headFlag, *heads, *trkNcl;
  OutBufs ob;
  OutBufs ob2;  // a second set of result arrays: replays alternate between the two
  int *lenHist, *stOrder;  // the sector fits' longest-first processing order
  int* trkTfBegin;
  double* coll;                       // interaction times of the batch
  int *memNext, *memPrev, *memPairs;  // membrane links and their pair count
};

GraphCaps graph_caps(long long maxClusters, int maxTFs, bool tight = false);
// Assigns the arena's pointers from base (null: only counts); returns bytes.
size_t graph_carve(GraphArena& A, char* base);
// Enqueues the whole pipeline on st (for stream capture).
void graph_enqueue(const GraphArena& A, const GeomConst* G, int nfBlock, bool nfStage, int sortThreads,
                   int forceFp64, cudaStream_t st, bool coopSearch = false, bool rowStep2 = false);

}  // namespace o2tpc
