// TPC clusterizer (Sec. 2.2: the raw ADC values are turned into hits before
// tracking) on the device, behind o2tpc_clusterize.
//
// Readings (the paper gives no algorithm): zero-suppressed digits sorted by
// (sector, row, time bin, pad); a peak is a digit with ADC >= 3 larger than
// each of its up to eight pad/time neighbours in the same row that come
// before it in that order and not smaller than each that comes after it; a
// peak's cluster is the 3 x 3 cells around it: Q = sum of ADC, centre of
// gravity of the cell centres (pad p spans [p, p + 1), bin t spans
// [t, t + 1)) in 1/64 units rounded half up in integers; one 12-byte record
// (u32 time64, u16 pad64, u16 min(Q, 65535), u8 row, u8 sector, u16 0) per
// peak, in the order of the peaks.  Exact integer arithmetic throughout.
//
// One thread per digit: the neighbours at the same time bin are the adjacent
// digits; those one bin earlier / later are found by a galloping search from
// the digit itself (they are close in the sorted order), then at most three
// entries are scanned.  Peaks are flagged, compacted in order with the warp
// ballots, and a second pass writes the records.
#include <cstdint>

#include "o2tpc.h"
#include "o2tpc_internal.cuh"
#include "o2tpc_kernels.cuh"

namespace o2tpc {

namespace {

constexpr int kPeakMin = 3;

__device__ inline unsigned long long dkey(uint8_t s, uint8_t r, uint32_t t, uint8_t p) {
  return ((unsigned long long)(s * kNRow + r) << 40) | ((unsigned long long)t << 8) | (unsigned long long)p;
}

// First index j in [lo, i) with k[j] >= key (galloping down from i).
__device__ inline long long gallop_down(const unsigned long long* __restrict__ k, long long i, unsigned long long key) {
  long long step = 1, hi = i, lo = i - 1;
  while (lo >= 0 && k[lo] >= key) {
    hi = lo;
    step <<= 1;
    lo = i - step;
  }
  if (lo < 0) lo = -1;
  // k[lo] < key (or lo = -1), k[hi] >= key (or hi = i)
  while (hi - lo > 1) {
    const long long m = (lo + hi) >> 1;
    if (k[m] >= key) hi = m;
    else lo = m;
  }
  return hi;
}

// First index j in (i, n] with k[j] >= key (galloping up from i).
__device__ inline long long gallop_up(const unsigned long long* __restrict__ k, long long n, long long i,
                                      unsigned long long key) {
  long long step = 1, lo = i, hi = i + 1;
  while (hi < n && k[hi] < key) {
    lo = hi;
    step <<= 1;
    hi = i + step;
  }
  if (hi > n) hi = n;
  while (hi - lo > 1) {
    const long long m = (lo + hi) >> 1;
    if (k[m] >= key) hi = m;
    else lo = m;
  }
  return hi;
}

// Peak test of digit i; for a peak also the 3 x 3 charge and position sums.
__device__ inline bool peak_of(const unsigned long long* __restrict__ k, const uint16_t* __restrict__ adc, long long n,
                               long long i, long long* q, long long* sp, long long* st) {
  const unsigned a = adc[i];
  if (a < (unsigned)kPeakMin) return false;
  const unsigned long long ki = k[i];
  const int p = (int)(ki & 0xff);
  const long long t = (long long)((ki >> 8) & 0xffffffffull);
  long long Q = a, SP = (long long)a * (64 * p + 32), ST = (long long)a * (64 * t + 32);
  // same time bin: the adjacent digits
  if (p > 0 && i > 0 && k[i - 1] == ki - 1) {
    const unsigned b = adc[i - 1];
    if (!(a > b)) return false;
    Q += b;
    SP += (long long)b * (64 * (p - 1) + 32);
    ST += (long long)b * (64 * t + 32);
  }
  if (p < 255 && i + 1 < n && k[i + 1] == ki + 1) {
    const unsigned b = adc[i + 1];
    if (!(a >= b)) return false;
    Q += b;
    SP += (long long)b * (64 * (p + 1) + 32);
    ST += (long long)b * (64 * t + 32);
  }
  const int p0 = p > 0 ? p - 1 : 0, p1 = p < 255 ? p + 1 : 255;
  // one bin earlier (all before i) and one bin later (all after i)
  for (int dt = -1; dt <= 1; dt += 2) {
    if (dt < 0 && t == 0) continue;
    const unsigned long long base = ki - (unsigned long long)p + ((unsigned long long)(t + dt) - (unsigned long long)t) * 256ull;
    const unsigned long long k0 = base + p0, k1 = base + p1;
    long long j = dt < 0 ? gallop_down(k, i, k0) : gallop_up(k, n, i, k0);
    for (; j < n && k[j] <= k1; ++j) {
      const unsigned b = adc[j];
      if (dt < 0 ? !(a > b) : !(a >= b)) return false;
      const int pj = (int)(k[j] & 0xff);
      Q += b;
      SP += (long long)b * (64 * pj + 32);
      ST += (long long)b * (64 * (t + dt) + 32);
    }
  }
  *q = Q;
  *sp = SP;
  *st = ST;
  return true;
}

}  // namespace

__global__ void k_clu_keys(long long n, const uint8_t* __restrict__ sector, const uint8_t* __restrict__ row,
                           const uint8_t* __restrict__ pad, const uint32_t* __restrict__ time,
                           unsigned long long* __restrict__ k, unsigned* __restrict__ err) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (sector[i] >= kNSec || row[i] >= kNRow || time[i] >= (1u << 24)) {
    atomicOr(err, kErrInput);
    k[i] = 0;
    return;
  }
  k[i] = dkey(sector[i], row[i], time[i], pad[i]);
}

__global__ void k_clu_flags(long long n, const unsigned long long* __restrict__ k, const uint16_t* __restrict__ adc,
                            int* __restrict__ flag, unsigned* __restrict__ err) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i > 0 && k[i] <= k[i - 1]) atomicOr(err, kErrInput);  // not strictly ascending
  long long q, sp, st;
  flag[i] = (*err & kErrInput) ? 0 : (peak_of(k, adc, n, i, &q, &sp, &st) ? 1 : 0);
}

__global__ void k_clu_records(const int* __restrict__ nPeaksDev, const int* __restrict__ peaks,
                              const unsigned long long* __restrict__ k, const uint16_t* __restrict__ adc, long long n,
                              uint8_t* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= *nPeaksDev) return;
  const long long i = peaks[c];
  long long q = 1, sp = 0, st = 0;
  peak_of(k, adc, n, i, &q, &sp, &st);
  const unsigned t64 = (unsigned)((2 * st + q) / (2 * q));
  const unsigned p64 = (unsigned)((2 * sp + q) / (2 * q));
  const unsigned ch = q > 65535 ? 65535u : (unsigned)q;
  const unsigned rr = (unsigned)(k[i] >> 40);
  uint8_t* r = out + 12 * (size_t)c;
  reinterpret_cast<uint32_t*>(r)[0] = t64;  // 12-byte records: 4-byte aligned
  reinterpret_cast<uint32_t*>(r)[1] = (p64 & 0xffffu) | (ch << 16);
  reinterpret_cast<uint32_t*>(r)[2] = (rr % kNRow) | ((rr / kNRow) << 8);
}

}  // namespace o2tpc

using namespace o2tpc;

extern "C" int o2tpc_clusterize(const o2tpc_digits* d, void* records, uint64_t cap, uint64_t* n_clusters,
                                void* stream) {
  if (!d || !n_clusters || (d->n > 0 && (!d->sector || !d->row || !d->pad || !d->time || !d->adc)) ||
      (cap > 0 && !records) || (reinterpret_cast<uintptr_t>(records) & 3))
    return O2TPC_EINVAL;
  *n_clusters = 0;
  if (d->n >= (1ull << 31)) return O2TPC_ETOOBIG;
  const long long n = (long long)d->n;
  if (n == 0) return O2TPC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nt = ballot_tiles(n);
  const size_t scanInts = (size_t)scan_scratch_ints(n + 8) + 64;
  const size_t bytes = 8 * (size_t)n + 4 * ((size_t)n + 1) + 8 * ((size_t)nt + 1) + 4 * (size_t)n + 4 * scanInts + 64;
  char* base = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return O2TPC_ENOMEM;
  }
  char* p = base;
  unsigned long long* k = reinterpret_cast<unsigned long long*>(p);
  p += 8 * (size_t)n;
  int* flag = reinterpret_cast<int*>(p);
  p += 4 * ((size_t)n + 1);
  int* tileCnt = reinterpret_cast<int*>(p);
  p += 4 * ((size_t)nt + 1);
  int* tileOff = reinterpret_cast<int*>(p);
  p += 4 * ((size_t)nt + 1);
  int* peaks = reinterpret_cast<int*>(p);
  p += 4 * (size_t)n;
  int* scratch = reinterpret_cast<int*>(p);
  p += 4 * scanInts;
  int* small = reinterpret_cast<int*>(p);  // [0] n, [1] peaks, [2] overflow, [3] error word
  int hs[4] = {(int)n, 0, 0, 0};
  int rc = O2TPC_OK;
  do {
    if (cudaMemcpyAsync(small, hs, sizeof(hs), cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = O2TPC_ECUDA; break; }
    unsigned* err = reinterpret_cast<unsigned*>(small + 3);
    const unsigned g = (unsigned)((n + 255) / 256);
    k_clu_keys<<<g, 256, 0, st>>>(n, d->sector, d->row, d->pad, d->time, k, err);
    k_clu_flags<<<g, 256, 0, st>>>(n, k, d->adc, flag, err);
    launch_ballot_count((int)n, small, flag, tileCnt, tileOff, small + 1, (int)n, small + 2, scratch, st);
    launch_ballot_compact((int)n, small, flag, tileOff, peaks, (int)n, small + 2, st);
    if (cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = O2TPC_ECUDA;
      break;
    }
    if (hs[3] & kErrInput) { rc = O2TPC_EINVAL; break; }
    *n_clusters = (uint64_t)hs[1];
    if ((uint64_t)hs[1] > cap) { rc = O2TPC_ETOOBIG; break; }
    if (hs[1] > 0) {
      k_clu_records<<<(hs[1] + 255) / 256, 256, 0, st>>>(small + 1, peaks, k, d->adc, n,
                                                          static_cast<uint8_t*>(records));
    }
    if (cudaGetLastError() != cudaSuccess) rc = O2TPC_ECUDA;
  } while (false);
  cudaFreeAsync(base, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == O2TPC_OK) rc = O2TPC_ECUDA;
  return rc;
}
