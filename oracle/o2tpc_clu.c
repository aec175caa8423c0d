/*
 * o2tpc_clu.c - oracle of the TPC clusterizer: raw ADC digits to clusters.
 *
 * TEST INFRASTRUCTURE ONLY (see o2tpc_oracle.h).  Plain C, single thread; it
 * shares no code with the CUDA path.
 *
 * Sec. 2.2: a clusterizing algorithm turns the raw ADC values into hits,
 * stored with no more bits than the TPC resolution needs.  The algorithm is
 * not given; the readings:
 *  - input: zero-suppressed digits (sector, row, pad, time bin, ADC), sorted
 *    strictly ascending by (sector, row, time bin, pad);
 *  - peak: a digit with ADC >= 3 that is larger than each of its up to eight
 *    pad/time neighbours in the same row coming before it in that order and
 *    not smaller than each neighbour coming after it (so a plateau of equal
 *    maxima yields one peak, its first digit);
 *  - cluster of a peak: over the 3 x 3 pad/time cells around it, the charge
 *    Q = sum of ADC and the centre of gravity of the cell centres (pad p spans
 *    [p, p + 1) pads, bin t spans [t, t + 1) bins) in 1/64 units, rounded half
 *    up in integer arithmetic: pad64 = floor((2 sum a (64 p + 32) + Q) / 2Q),
 *    likewise time64;
 *  - output: one 12-byte cluster record per peak (u32 time64, u16 pad64,
 *    u16 min(Q, 65535), u8 row, u8 sector, u16 0), in the order of the peaks.
 */
#include <stdint.h>
#include <stdlib.h>

#include "o2tpc_oracle.h"

#define U_NROW 152
#define U_PEAK_MIN 3

static uint64_t u_key(uint8_t s, uint8_t r, uint32_t t, uint8_t p) {
  return ((uint64_t)(s * U_NROW + r) << 40) | ((uint64_t)t << 8) | (uint64_t)p;
}

static int64_t u_find(const uint64_t* k, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) / 2;
    if (k[m] < key) lo = m + 1;
    else hi = m;
  }
  return (lo < n && k[lo] == key) ? lo : -1;
}

int64_t oracle_clusterize(int64_t n, const uint8_t* sector, const uint8_t* row, const uint8_t* pad,
                          const uint32_t* time, const uint16_t* adc, uint8_t** out) {
  uint64_t* k = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  for (int64_t i = 0; i < n; ++i) {
    if (sector[i] >= 36 || row[i] >= U_NROW || time[i] >= (1u << 24)) { free(k); return -1; }
    k[i] = u_key(sector[i], row[i], time[i], pad[i]);
    if (i > 0 && k[i] <= k[i - 1]) { free(k); return -1; }
  }
  uint8_t* rec = (uint8_t*)malloc(12 * (size_t)n + 12);
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (adc[i] < U_PEAK_MIN) continue;
    int peak = 1;
    int64_t q = 0, sp = 0, st = 0;
    for (int dt = -1; dt <= 1 && peak; ++dt)
      for (int dp = -1; dp <= 1; ++dp) {
        int64_t t = (int64_t)time[i] + dt, p = (int64_t)pad[i] + dp;
        if (t < 0 || p < 0 || p > 255) continue;
        int64_t j = (dt == 0 && dp == 0) ? i : u_find(k, n, u_key(sector[i], row[i], (uint32_t)t, (uint8_t)p));
        if (j < 0) continue;
        if (j < i && !(adc[i] > adc[j])) { peak = 0; break; }
        if (j > i && !(adc[i] >= adc[j])) { peak = 0; break; }
        q += adc[j];
        sp += (int64_t)adc[j] * (64 * p + 32);
        st += (int64_t)adc[j] * (64 * t + 32);
      }
    if (!peak) continue;
    uint32_t t64 = (uint32_t)((2 * st + q) / (2 * q));
    uint32_t p64 = (uint32_t)((2 * sp + q) / (2 * q));
    uint32_t ch = q > 65535 ? 65535u : (uint32_t)q;
    uint8_t* r = rec + 12 * nc;
    r[0] = (uint8_t)t64; r[1] = (uint8_t)(t64 >> 8); r[2] = (uint8_t)(t64 >> 16); r[3] = (uint8_t)(t64 >> 24);
    r[4] = (uint8_t)p64; r[5] = (uint8_t)(p64 >> 8);
    r[6] = (uint8_t)ch; r[7] = (uint8_t)(ch >> 8);
    r[8] = row[i]; r[9] = sector[i]; r[10] = 0; r[11] = 0;
    ++nc;
  }
  free(k);
  *out = rec;
  return nc;
}
