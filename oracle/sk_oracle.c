/*
 * CPU oracle for the SparseStack sketch Y = S*A with FP32 or emulated FP16 accumulation.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py may load this library. The CUDA product path never calls it.
 * It shares no code with the CUDA sources: every generator, rounding routine and loop here
 * is written independently from the published definitions cited below.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * -ffp-contract=off is required: the FP32 sequences below must round after every operation.
 *
 * What follows, and the passage each part restates:
 *   - SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 *     OOPSLA 2014): the counter-based source of the sketch pattern.
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *     SC'11): the rounding random bits.
 *   - SparseStack operator S (paper Sec. 2.2, Definition of SparseStack; Sec. 4.1 for the block
 *     ranges [j d/zeta, (j+1) d/zeta) and the 1/sqrt(zeta) value scaling).
 *   - IEEE 754 binary16 rounding (round-to-nearest-even, toward -inf, toward +inf) and binary16
 *     addition, written from the format definition.
 *   - The three quantizers of paper Sec. 4.2: round-to-nearest (default hardware conversion),
 *     exact stochastic rounding and dithered rounding, with the two constants the paper leaves
 *     open fixed as: the scale of the 24-bit random integer that makes the uniform u, 2^-24, and
 *     the dither amplitude factor (noise = (u - 1/2) * x * factor, about one binary16 ulp), 2^-10.
 *   - The FP64 sketch (dense S times A semantics of Sec. 4.1) and the canonical-order FP32/FP16
 *     accumulation: per output, chunk partials in FP32 over ascending rows, scaled, quantized,
 *     then accumulated in ascending chunk order (FP16 adds are round-to-nearest-even).
 *
 * Parity status: every function here is pinned by tests in tests/test_oracle_*.py
 * (published test vectors, closed forms, brute force, invariants). None is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define SKO_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------- SplitMix64 */
static const uint64_t SKO_GOLDEN_GAMMA = 0x9E3779B97F4A7C15ULL;

/* The SplitMix64 output function (Stafford variant 13 finalizer, as used by SplitMix64). */
SKO_EXPORT uint64_t sko_splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The n-th output (n >= 1) of a SplitMix64 generator whose state starts at `seed`:
 * the state advances by the golden gamma before every output. */
SKO_EXPORT uint64_t sko_splitmix64_nth(uint64_t seed, uint64_t n) {
  return sko_splitmix64_mix(seed + n * SKO_GOLDEN_GAMMA);
}

/* ---------------------------------------------------------------- Philox4x32-10 */
static void sko_mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

SKO_EXPORT void sko_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    sko_mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    sko_mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The uniform u in [0,1) used to round contribution t of output (r, c):
 * word (c mod 4) of Philox4x32-10 with key (lo32 seed, hi32 seed) and
 * counter (r, floor(c/4), lo32 t, hi32 t); u = (word & 0xFFFFFF) * 2^-24 (paper Sec. 4.2). */
SKO_EXPORT float sko_uniform(uint64_t seed, int64_t r, int64_t c, int64_t t) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(c >> 2), (uint32_t)(uint64_t)t, (uint32_t)((uint64_t)t >> 32)};
  uint32_t w[4];
  sko_philox4x32_10(ctr, key, w);
  uint32_t bits = w[c & 3] & 0x00FFFFFFu;
  return (float)bits * (1.0f / 16777216.0f);
}

/* ---------------------------------------------------------------- S pattern */
/* Row i, block j of a SparseStack with d rows, k blocks of B = d/k rows:
 * the SplitMix64 output number (i*ceil(k/2) + floor(j/2) + 1) of the generator started at `seed`
 * supplies 64 bits; block j uses its high 32-bit half when j is even, the low half when j is odd.
 * With w that 32-bit word: target s = j*B + floor(w*B / 2^32), sign = -1 if (w & 1) else +1. */
SKO_EXPORT void sko_target(uint64_t seed, int64_t i, int32_t k, int64_t B, int32_t j, int64_t* s, int* neg) {
  uint64_t kp = (uint64_t)((k + 1) / 2);
  uint64_t h = sko_splitmix64_nth(seed, (uint64_t)i * kp + (uint64_t)(j / 2) + 1u);
  uint32_t w = (j % 2 == 0) ? (uint32_t)(h >> 32) : (uint32_t)h;
  *s = (int64_t)j * B + (int64_t)(((uint64_t)w * (uint64_t)B) >> 32);
  *neg = (int)(w & 1u);
}

/* rows[(i-i0)*k + j] = s_ij, signs[...] = +1 / -1 for i in [i0, i0+cnt). */
SKO_EXPORT void sko_s_pattern(int64_t d, int32_t k, uint64_t seed, int64_t i0, int64_t cnt, int64_t* rows,
                              int8_t* signs) {
  int64_t B = d / k;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < cnt; ++q) {
    for (int32_t j = 0; j < k; ++j) {
      int64_t s;
      int neg;
      sko_target(seed, i0 + q, k, B, j, &s, &neg);
      rows[q * k + j] = s;
      signs[q * k + j] = neg ? (int8_t)-1 : (int8_t)1;
    }
  }
}

/* ---------------------------------------------------------------- binary16 */
/* Exact value of a binary16 bit pattern as a double. */
SKO_EXPORT double sko_half_to_double(uint16_t h) {
  int sign = (h >> 15) & 1;
  int e = (h >> 10) & 0x1F;
  int f = h & 0x3FF;
  double v;
  if (e == 0x1F) {
    v = f ? NAN : INFINITY;
  } else if (e == 0) {
    v = ldexp((double)f, -24);
  } else {
    v = ldexp((double)(f + 1024), e - 25);
  }
  return sign ? -v : v;
}

/* Round a double to binary16. mode 0: nearest, ties to even; 1: toward -inf; 2: toward +inf. */
SKO_EXPORT uint16_t sko_round_to_half(double x, int mode) {
  if (isnan(x)) return 0x7E00u;
  uint16_t sgn = signbit(x) ? 0x8000u : 0u;
  double a = fabs(x);
  if (a == 0.0) return sgn;
  /* Magnitude rounding direction: 0 nearest-even, 1 toward zero, 2 away from zero. */
  int mag_mode;
  if (mode == 0) mag_mode = 0;
  else if (mode == 1) mag_mode = sgn ? 2 : 1;
  else mag_mode = sgn ? 1 : 2;
  if (isinf(a)) return (uint16_t)(sgn | 0x7C00u);
  int E2;
  (void)frexp(a, &E2); /* a = f * 2^E2, f in [0.5, 1) => floor(log2 a) = E2 - 1 */
  int e = E2 - 1;
  if (e > 15) {
    /* Beyond the largest finite binade: nearest and away give inf; toward zero gives max. */
    return (uint16_t)(sgn | (mag_mode == 1 ? 0x7BFFu : 0x7C00u));
  }
  int qexp = (e < -14) ? -24 : (e - 10); /* quantum 2^qexp */
  double N = ldexp(a, -qexp);           /* exact: scaling by a power of two */
  double nf = floor(N);
  double frac = N - nf; /* exact */
  double n = nf;
  if (mag_mode == 0) {
    if (frac > 0.5) n = nf + 1.0;
    else if (frac == 0.5) n = (fmod(nf, 2.0) == 0.0) ? nf : nf + 1.0;
  } else if (mag_mode == 2) {
    if (frac > 0.0) n = nf + 1.0;
  }
  double M = ldexp(n, qexp); /* rounded magnitude, exact */
  if (M == 0.0) return sgn;
  if (M >= 65536.0) return (uint16_t)(sgn | 0x7C00u);
  int E2m;
  (void)frexp(M, &E2m);
  int em = E2m - 1;
  uint16_t bits;
  if (em < -14) {
    bits = (uint16_t)ldexp(M, 24); /* subnormal: M = bits * 2^-24 */
  } else {
    uint32_t mant = (uint32_t)ldexp(M, 10 - em) - 1024u;
    bits = (uint16_t)(((uint32_t)(em + 15) << 10) | mant);
  }
  return (uint16_t)(sgn | bits);
}

/* binary16 + binary16, rounded to nearest even. The double sum of two binary16 values is exact
 * (their significands span at most 40 bits), so one rounding of it is the IEEE result. */
SKO_EXPORT uint16_t sko_half_add(uint16_t a, uint16_t b) {
  return sko_round_to_half(sko_half_to_double(a) + sko_half_to_double(b), 0);
}

/* ---------------------------------------------------------------- bfloat16 */
/* bfloat16 (paper Sec. 4.2 names it beside FP16 as a 16-bit reduction target): the upper 16 bits of
 * a binary32, i.e. 8 significant bits with binary32's exponent range. */

/* Exact value of a bfloat16 bit pattern as a double. */
SKO_EXPORT double sko_bf16_to_double(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* Round a double to bfloat16, nearest with ties to even (same construction as sko_round_to_half:
 * scale by the quantum of the binade, round the integer part, scale back). */
SKO_EXPORT uint16_t sko_round_to_bf16(double x) {
  if (isnan(x)) return 0x7FC0u;
  uint16_t sgn = signbit(x) ? 0x8000u : 0u;
  double a = fabs(x);
  if (a == 0.0) return sgn;
  if (isinf(a)) return (uint16_t)(sgn | 0x7F80u);
  int E2;
  (void)frexp(a, &E2);
  int e = E2 - 1;                         /* a in [2^e, 2^(e+1)) */
  if (e > 127) return (uint16_t)(sgn | 0x7F80u);
  int qexp = (e < -126) ? -133 : (e - 7); /* quantum: 7 fraction bits, subnormal quantum 2^-133 */
  double N = ldexp(a, -qexp);
  double nf = floor(N);
  double frac = N - nf;
  double n = nf;
  if (frac > 0.5) n = nf + 1.0;
  else if (frac == 0.5) n = (fmod(nf, 2.0) == 0.0) ? nf : nf + 1.0;
  double M = ldexp(n, qexp);
  if (M == 0.0) return sgn;
  if (M >= 0x1p128) return (uint16_t)(sgn | 0x7F80u);
  int E2m;
  (void)frexp(M, &E2m);
  int em = E2m - 1;
  uint16_t bits;
  if (em < -126) {
    bits = (uint16_t)ldexp(M, 133); /* subnormal: M = bits * 2^-133 */
  } else {
    uint32_t mant = (uint32_t)ldexp(M, 7 - em) - 128u;
    bits = (uint16_t)(((uint32_t)(em + 127) << 7) | mant);
  }
  return (uint16_t)(sgn | bits);
}

/* bfloat16 + bfloat16, rounded to nearest even. The double sum is exact unless the exponents differ
 * by more than 45; then the smaller operand is far below half an ulp of the larger, and the exact
 * and the double sum both round to the larger operand, so one rounding of the double sum is the
 * correctly rounded result. */
SKO_EXPORT uint16_t sko_bf16_add(uint16_t a, uint16_t b) {
  return sko_round_to_bf16(sko_bf16_to_double(a) + sko_bf16_to_double(b));
}

/* Array forms of the conversions and additions above (element-wise, threads over the elements), for
 * the exhaustive comparisons of the tests: every binary32 pattern rounded to binary16 (mode as for
 * sko_round_to_half) or bfloat16, and every pair of 16-bit patterns added. No new arithmetic. */
SKO_EXPORT void sko_round_to_half_f32_array(const float* x, int64_t n, int mode, uint16_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = sko_round_to_half((double)x[i], mode);
}

SKO_EXPORT void sko_half_add_array(const uint16_t* a, const uint16_t* b, int64_t n, uint16_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = sko_half_add(a[i], b[i]);
}

SKO_EXPORT void sko_round_to_bf16_f32_array(const float* x, int64_t n, uint16_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = sko_round_to_bf16((double)x[i]);
}

SKO_EXPORT void sko_bf16_add_array(const uint16_t* a, const uint16_t* b, int64_t n, uint16_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = sko_bf16_add(a[i], b[i]);
}

/* ---------------------------------------------------------------- quantizers (paper Sec. 4.2) */
enum { SKO_FP32 = 0, SKO_FP16_RN = 1, SKO_FP16_SR = 2, SKO_FP16_DITHER = 3, SKO_BF16_RN = 4 };

/* 16-bit addition of the rule's format (binary16 or bfloat16), round to nearest even. */
static uint16_t sko_add16(uint16_t a, uint16_t b, int rule) {
  return (rule == SKO_BF16_RN) ? sko_bf16_add(a, b) : sko_half_add(a, b);
}

/* Rules that draw no random bits. */
static int sko_rule_is_rn(int rule) { return rule == SKO_FP16_RN || rule == SKO_BF16_RN; }

/* x: the FP32 value to store; u: uniform in [0,1). Every FP32 operation rounds (no contraction). */
SKO_EXPORT uint16_t sko_quantize(float x, float u, int rule) {
  if (rule == SKO_FP16_RN) {
    return sko_round_to_half((double)x, 0);
  }
  if (rule == SKO_FP16_SR) {
    /* Sec. 4.2, exact stochastic rounding: the upper binary16 neighbour with probability
     * (x - lower) / (upper - lower), decided by comparing u times the gap with the excess of x over
     * the lower neighbour. Both differences are exact in FP32 (the gap is a power of two; the excess
     * follows from Sterbenz's lemma); the product u * gap is exact too. */
    uint16_t lower = sko_round_to_half((double)x, 1);
    uint16_t upper = sko_round_to_half((double)x, 2);
    float lo = (float)sko_half_to_double(lower);
    float gap = (float)sko_half_to_double(upper) - lo;
    float excess = x - lo;
    return (u * gap < excess) ? upper : lower;
  }
  if (rule == SKO_BF16_RN) {
    return sko_round_to_bf16((double)x);
  }
  if (rule == SKO_FP16_DITHER) {
    /* Sec. 4.2, dithered rounding: zero-mean uniform noise of amplitude x * 2^-10 added in FP32,
     * then round to nearest even. */
    const float factor = 1.0f / 1024.0f; /* 2^-10 */
    float centered = u - 0.5f;
    float amplitude = x * factor;
    float noise = centered * amplitude;
    float y = x + noise;
    return sko_round_to_half((double)y, 0);
  }
  return 0;
}

/* ---------------------------------------------------------------- sketches */
/* FP64 sketch: Y64[r*n + c] = (1/sqrt(k)) * sum over (i, j) with s_ij = r of sign_ij * A[i*lda + c]. */
SKO_EXPORT void sko_sketch_f64(const float* A, int64_t lda, int64_t m, int64_t n, int64_t d, int32_t k,
                               uint64_t seed, double* Y) {
  int64_t B = d / k;
  double inv = 1.0 / sqrt((double)k);
  memset(Y, 0, sizeof(double) * (size_t)(d * n));
  /* Parallel over blocks: block j writes only rows [jB, (j+1)B). */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < k; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      int64_t s;
      int neg;
      sko_target(seed, i, k, B, j, &s, &neg);
      const float* a = A + i * lda;
      double* y = Y + s * n;
      for (int64_t c = 0; c < n; ++c) y[c] += neg ? -(double)a[c] : (double)a[c];
    }
  }
  for (int64_t q = 0; q < d * n; ++q) Y[q] *= inv;
}

/* Canonical-order accumulation for `rule` with chunk length R rows (R >= 1).
 * For output (r, c), r in block j: for every chunk t = floor(i/R) holding at least one row i with
 * s_ij = r, in ascending t: P = FP32 sum from +0 of sign*A[i,c] over those rows in ascending i;
 * x = fl32(scale * P) with scale = fl32(1/sqrt(k)); then
 *   FP32 rule:  Y = fl32(Y + x);
 *   FP16 rules: Y = RN16(Y + Q(x, u(r, c, t)));
 *   BF16 rule:  Y = RNbf16(Y + RNbf16(x)).
 * Y starts at +0. Y is float[d*n] for the FP32 rule, 16-bit patterns uint16[d*n] otherwise. */
SKO_EXPORT void sko_sketch_canonical(const float* A, int64_t lda, int64_t m, int64_t n, int64_t d, int32_t k,
                                     uint64_t seed, int rule, int64_t R, void* Yout) {
  int64_t B = d / k;
  float scale = (float)(1.0 / sqrt((double)k));
  float* Y32 = (float*)Yout;
  uint16_t* Y16 = (uint16_t*)Yout;
  if (rule == SKO_FP32) {
    for (int64_t q = 0; q < d * n; ++q) Y32[q] = 0.0f;
  } else {
    for (int64_t q = 0; q < d * n; ++q) Y16[q] = 0u;
  }
  /* Targets of every row for every block, computed once. */
  int64_t* tgt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m * k));
  int8_t* sg = (int8_t*)malloc((size_t)(m * k));
  sko_s_pattern(d, k, seed, 0, m, tgt, sg);
  /* Each (block j, column c) is independent: it owns outputs (jB..jB+B-1, c). */
#pragma omp parallel
  {
    float* P = (float*)malloc(sizeof(float) * (size_t)B);
    unsigned char* touched = (unsigned char*)calloc((size_t)B, 1);
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)B);
#pragma omp for schedule(dynamic, 1)
    for (int64_t jc = 0; jc < (int64_t)k * n; ++jc) {
      int32_t j = (int32_t)(jc / n);
      int64_t c = jc % n;
      for (int64_t t0 = 0; t0 < m; t0 += R) {
        int64_t t = t0 / R;
        int64_t t1 = (t0 + R < m) ? t0 + R : m;
        int64_t nl = 0;
        for (int64_t i = t0; i < t1; ++i) {
          int64_t sl = tgt[i * k + j] - (int64_t)j * B;
          if (!touched[sl]) {
            touched[sl] = 1;
            P[sl] = 0.0f;
            list[nl++] = sl;
          }
          float a = A[i * lda + c];
          float v = (sg[i * k + j] < 0) ? -a : a;
          P[sl] = P[sl] + v;
        }
        for (int64_t q = 0; q < nl; ++q) {
          int64_t sl = list[q];
          int64_t r = (int64_t)j * B + sl;
          float x = scale * P[sl];
          if (rule == SKO_FP32) {
            Y32[r * n + c] = Y32[r * n + c] + x;
          } else {
            float u = sko_rule_is_rn(rule) ? 0.0f : sko_uniform(seed, r, c, t);
            uint16_t qv = sko_quantize(x, u, rule);
            Y16[r * n + c] = sko_add16(Y16[r * n + c], qv, rule);
          }
          touched[sl] = 0;
        }
      }
    }
    free(P);
    free(touched);
    free(list);
  }
  free(tgt);
  free(sg);
}

/* The same two results at selected outputs only, for matrices too large for the full oracle.
 * out64[q] = FP64 value and outc[q] = canonical value (float, or the 16-bit pattern in the low 16 bits
 * of a uint32) at output (rs[q], cs[q]). Every row of A is scanned once per selected output. */
SKO_EXPORT void sko_sketch_sampled(const float* A, int64_t lda, int64_t m, int64_t n, int64_t d, int32_t k,
                                   uint64_t seed, int rule, int64_t R, int64_t cnt, const int64_t* rs,
                                   const int64_t* cs, double* out64, uint32_t* outc) {
  int64_t B = d / k;
  float scale = (float)(1.0 / sqrt((double)k));
  double inv = 1.0 / sqrt((double)k);
  (void)n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < cnt; ++q) {
    int64_t r = rs[q], c = cs[q];
    int32_t j = (int32_t)(r / B);
    double acc64 = 0.0;
    float Y32 = 0.0f;
    uint16_t Y16 = 0u;
    float P = 0.0f;
    int64_t cur_t = -1;
    for (int64_t i = 0; i < m; ++i) {
      int64_t s;
      int neg;
      sko_target(seed, i, k, B, j, &s, &neg);
      if (s != r) continue;
      float a = A[i * lda + c];
      acc64 += neg ? -(double)a : (double)a;
      int64_t t = i / R;
      if (t != cur_t) {
        if (cur_t >= 0) {
          float x = scale * P;
          if (rule == SKO_FP32) {
            Y32 = Y32 + x;
          } else {
            float u = sko_rule_is_rn(rule) ? 0.0f : sko_uniform(seed, r, c, cur_t);
            Y16 = sko_add16(Y16, sko_quantize(x, u, rule), rule);
          }
        }
        cur_t = t;
        P = 0.0f;
      }
      P = P + (neg ? -a : a);
    }
    if (cur_t >= 0) {
      float x = scale * P;
      if (rule == SKO_FP32) {
        Y32 = Y32 + x;
      } else {
        float u = sko_rule_is_rn(rule) ? 0.0f : sko_uniform(seed, r, c, cur_t);
        Y16 = sko_add16(Y16, sko_quantize(x, u, rule), rule);
      }
    }
    out64[q] = acc64 * inv;
    if (rule == SKO_FP32) {
      uint32_t bits;
      memcpy(&bits, &Y32, 4);
      outc[q] = bits;
    } else {
      outc[q] = Y16;
    }
  }
}

/* Number of OpenMP threads the oracle uses (for reporting). */
SKO_EXPORT int sko_num_threads(void) {
  int nt = 1;
#pragma omp parallel
  {
#pragma omp single
    {
#ifdef _OPENMP
      nt = omp_get_num_threads();
#endif
    }
  }
  return nt;
}
