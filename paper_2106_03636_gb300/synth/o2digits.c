/*
 * o2digits.c - raw ADC digits for a TF's clusters (input generator for the
 * clusterizer; no clusterizer arithmetic here).
 *
 * Each cluster of a fixed-format TF deposits a charge Q = 20 + charge / 6 ADC
 * counts on the pad x time-bin grid of its pad row with a two-dimensional
 * Gaussian profile (sigma_pad pads, sigma_time bins; pad p spans [p, p + 1)
 * pads from the pad-plane edge, bin t spans [t, t + 1) bins, as the cluster
 * format's pad64 / time64 do), over the 5 x 5 cells around it.  Deposits of
 * all clusters are summed per cell, Gaussian noise of sigma `noise` counts is
 * added (drawn from a counter-based generator keyed by the cell, so the
 * result does not depend on the cluster order), the sum is rounded, capped at
 * 1023 and zero-suppressed below `threshold`.  The digits come out sorted by
 * (sector, row, time bin, pad).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define D_NROW 152

typedef struct {
  uint64_t key; /* sector * 152 + row << 40 | time << 8 | pad */
  float v;
} d_dep;

static uint64_t d_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double d_gauss(uint64_t h) { /* Box-Muller on two 53-bit uniforms */
  double u1 = ((double)(d_mix(h) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((double)(d_mix(h ^ 0xD1B54A32D192ED03ull) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static double d_cdf(double x) { return 0.5 * erfc(-x * 0.70710678118654752); }

/* LSD radix sort of deposits by key (7 passes of 8 bits cover the 53 used
 * bits), stable; the result ends in a. */
static void d_sort(d_dep* a, int64_t n) {
  d_dep* src = a;
  d_dep* dst = (d_dep*)malloc(sizeof(d_dep) * (size_t)(n + 1));
  d_dep* other = dst;
  for (int pass = 0; pass < 7; ++pass) {
    int sh = 8 * pass;
    int64_t cnt[257];
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; ++i) cnt[((src[i].key >> sh) & 0xff) + 1]++;
    for (int k = 0; k < 256; ++k) cnt[k + 1] += cnt[k];
    for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i].key >> sh) & 0xff]++] = src[i];
    d_dep* t = src; src = dst; dst = t;
  }
  if (src != a) memcpy(a, src, sizeof(d_dep) * (size_t)n);
  free(other);
}

int64_t o2dig_run(int64_t n, const uint8_t* packed, uint64_t seed, double sig_pad, double sig_time, double noise,
                  int32_t threshold, uint8_t** sector, uint8_t** row, uint8_t** pad, uint32_t** time,
                  uint16_t** adc) {
  d_dep* dep = (d_dep*)malloc(sizeof(d_dep) * (size_t)(25 * n + 1));
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const uint8_t* r = packed + 12 * i;
    uint32_t t64 = (uint32_t)r[0] | ((uint32_t)r[1] << 8) | ((uint32_t)r[2] << 16) | ((uint32_t)r[3] << 24);
    uint32_t p64 = (uint32_t)r[4] | ((uint32_t)r[5] << 8);
    uint32_t ch = (uint32_t)r[6] | ((uint32_t)r[7] << 8);
    uint32_t rw = r[8], sec = r[9];
    double pc = p64 / 64.0, tc = t64 / 64.0, q = 20.0 + ch / 6.0;
    int64_t p0 = (int64_t)floor(pc), t0 = (int64_t)floor(tc);
    for (int64_t dt = -2; dt <= 2; ++dt) {
      int64_t t = t0 + dt;
      if (t < 0 || t >= (1ll << 32)) continue;
      double ft = d_cdf((t + 1 - tc) / sig_time) - d_cdf((t - tc) / sig_time);
      for (int64_t dp = -2; dp <= 2; ++dp) {
        int64_t p = p0 + dp;
        if (p < 0 || p > 255) continue;
        double fp = d_cdf((p + 1 - pc) / sig_pad) - d_cdf((p - pc) / sig_pad);
        dep[m].key = ((uint64_t)(sec * D_NROW + rw) << 40) | ((uint64_t)t << 8) | (uint64_t)p;
        dep[m].v = (float)(q * ft * fp);
        ++m;
      }
    }
  }
  d_sort(dep, m);
  int64_t nd = 0;
  uint8_t* S = (uint8_t*)malloc((size_t)m + 1);
  uint8_t* R = (uint8_t*)malloc((size_t)m + 1);
  uint8_t* P = (uint8_t*)malloc((size_t)m + 1);
  uint32_t* T = (uint32_t*)malloc(4 * (size_t)m + 4);
  uint16_t* A = (uint16_t*)malloc(2 * (size_t)m + 2);
  for (int64_t i = 0; i < m;) {
    uint64_t k = dep[i].key;
    double v = 0.0;
    while (i < m && dep[i].key == k) v += dep[i++].v;
    v += noise * d_gauss(seed ^ d_mix(k));
    double a = floor(v + 0.5);
    if (a < threshold) continue;
    if (a > 1023) a = 1023;
    uint32_t rr = (uint32_t)(k >> 40);
    S[nd] = (uint8_t)(rr / D_NROW);
    R[nd] = (uint8_t)(rr % D_NROW);
    T[nd] = (uint32_t)((k >> 8) & 0xffffffffull);
    P[nd] = (uint8_t)(k & 0xff);
    A[nd] = (uint16_t)a;
    ++nd;
  }
  free(dep);
  *sector = S; *row = R; *pad = P; *time = T; *adc = A;
  return nd;
}

void o2dig_free(void* p) { free(p); }
