// Device primitives of the sketch kernels: the counter-based S generator, Philox4x32-10 for the
// rounding bits, and the three FP16 quantizers of paper Sec. 4.2.
//
// Every FP32 operation whose rounding matters is written with an explicit _rn intrinsic so that
// nvcc cannot contract it into an FMA: the deterministic modes must reproduce the canonical order
// bit for bit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace sk {

// ------------------------------------------------------------------ SplitMix64
// Steele, Lea & Flood, "Fast splittable pseudorandom number generators" (OOPSLA 2014): the state
// advances by the golden-ratio increment and each output is the state passed through the 64-bit
// finalizer below.
__device__ __forceinline__ uint64_t splitmix_finalize(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// SplitMix64 state increment (the golden-ratio gamma).
constexpr uint64_t kSplitMixGamma = 0x9E3779B97F4A7C15ull;

// Output number `idx` (idx >= 1) of the SplitMix64 stream started at `seed`.
__device__ __forceinline__ uint64_t splitmix_output(uint64_t seed, uint64_t idx) {
  return splitmix_finalize(seed + idx * kSplitMixGamma);
}

// The 64 bits serving blocks 2p and 2p+1 of input row i: stream output i*kp + p + 1, kp = ceil(k/2).
__device__ __forceinline__ uint64_t row_pair_bits(uint64_t seed, uint64_t i, uint32_t kp, uint32_t p) {
  return splitmix_output(seed, i * (uint64_t)kp + (uint64_t)p + 1ull);
}

// 32-bit word of block j from the 64 bits of its block pair: even j -> high half, odd j -> low half.
__device__ __forceinline__ uint32_t block_word(uint64_t bits, uint32_t j) {
  return (j & 1u) ? (uint32_t)bits : (uint32_t)(bits >> 32);
}

// Row offset inside block j (0 <= s < B) from the block's word: Lemire's multiply-shift,
// floor(w * B / 2^32). Sign bit: bit 0 of the word (1 -> negative).
__device__ __forceinline__ uint32_t word_to_slot(uint32_t w, uint32_t B) { return __umulhi(w, B); }

// ------------------------------------------------------------------ element types of A
// A arrives as FP32, binary16 or bfloat16; 16-bit values convert to FP32 exactly as they are read,
// so the arithmetic after the load is the FP32 path's.
enum AType { kAF32 = 0, kAF16 = 1, kABF16 = 2 };

template <typename TA>
__device__ __forceinline__ float a_to_f32(TA v) {
  if constexpr (std::is_same<TA, __half>::value) return __half2float(v);
  else if constexpr (std::is_same<TA, __nv_bfloat16>::value) return __bfloat162float(v);
  else return v;
}

// Read-only load of one element of A (through the non-coherent cache) converted to FP32.
template <typename TA>
__device__ __forceinline__ float ld_a(const TA* p) {
  if constexpr (std::is_same<TA, float>::value) return __ldg(p);
  else return a_to_f32(__ldg(p));
}

// One element of A of run-time type `a_type` (slow paths: deterministic and literal kernels).
__device__ __forceinline__ float ld_a_any(const void* A, int32_t a_type, int64_t idx) {
  if (a_type == kAF16) return ld_a(static_cast<const __half*>(A) + idx);
  if (a_type == kABF16) return ld_a(static_cast<const __nv_bfloat16*>(A) + idx);
  return ld_a(static_cast<const float*>(A) + idx);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                          uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi_b ^ c1 ^ k0;
    const uint32_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0;
    c1 = lo_b;
    c2 = n2;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return {c0, c1, c2, c3};
}

// Four uniforms in [0,1) for output row r, columns 4q..4q+3, contribution t. The key is the seed,
// the counter (r, q, lo32 t, hi32 t). Each uses the low 24 bits of its word times 2^-24.
__device__ __forceinline__ void uniforms4(uint64_t seed, uint32_t r, uint32_t q, uint64_t t, float u[4]) {
  const u32x4 w = philox10(r, q, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)seed, (uint32_t)(seed >> 32));
  const float s = 5.9604644775390625e-08f;  // 2^-24
  u[0] = __fmul_rn(__uint2float_rn(w.x & 0xFFFFFFu), s);
  u[1] = __fmul_rn(__uint2float_rn(w.y & 0xFFFFFFu), s);
  u[2] = __fmul_rn(__uint2float_rn(w.z & 0xFFFFFFu), s);
  u[3] = __fmul_rn(__uint2float_rn(w.w & 0xFFFFFFu), s);
}

// ------------------------------------------------------------------ FP16 quantizers (paper Sec. 4.2)
enum Rule : int { kFP32 = 0, kRN = 1, kSR = 2, kDither = 3, kBF16 = 4 };

// Exact stochastic rounding: upper neighbour with probability (x - rd) / (ru - rd).
__device__ __forceinline__ __half quant_sr(float x, float u) {
  const __half lo = __float2half_rd(x);
  const __half hi = __float2half_ru(x);
  const float flo = __half2float(lo);
  const float span = __fsub_rn(__half2float(hi), flo);
  const float off = __fsub_rn(x, flo);
  return (__fmul_rn(u, span) < off) ? hi : lo;
}

// Non-subtractive dither: zero-mean uniform noise of amplitude x * 2^-10 (about one binary16 ulp),
// then round to nearest even.
__device__ __forceinline__ __half quant_dither(float x, float u) {
  const float noise = __fmul_rn(__fsub_rn(u, 0.5f), __fmul_rn(x, 0.0009765625f));
  return __float2half_rn(__fadd_rn(x, noise));
}

template <int RULE>
__device__ __forceinline__ __half quantize(float x, float u) {
  if (RULE == kSR) return quant_sr(x, u);
  if (RULE == kDither) return quant_dither(x, u);
  return __float2half_rn(x);
}

// ------------------------------------------------------------------ 16-bit rules as bit patterns
// The 16-bit rules store Y as binary16 (FP16 rules) or bfloat16 (kBF16: round to nearest even, the
// BF16 reduction target of paper Sec. 4.2). Values travel as their 16-bit patterns.

// Rules whose quantizer draws uniforms (the others round to nearest).
template <int RULE>
__device__ __forceinline__ constexpr bool rule_draws_bits() {
  return RULE == kSR || RULE == kDither;
}

template <int RULE>
__device__ __forceinline__ uint16_t quantize16(float x, float u) {
  if (RULE == kBF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  return __half_as_ushort(quantize<RULE>(x, u));
}

// a + b in the rule's 16-bit format, rounded to nearest even.
template <int RULE>
__device__ __forceinline__ uint16_t add16(uint16_t a, uint16_t b) {
  if (RULE == kBF16) return __bfloat16_as_ushort(__hadd(__ushort_as_bfloat16(a), __ushort_as_bfloat16(b)));
  return __half_as_ushort(__hadd(__ushort_as_half(a), __ushort_as_half(b)));
}

// Atomic y[0] += q0, y[1] += q1 (one packed 32-bit atomic; y 4-byte aligned), and the scalar form.
template <int RULE>
__device__ __forceinline__ void atomic_add16x2(uint16_t* y, uint16_t q0, uint16_t q1) {
  if (RULE == kBF16) {
    atomicAdd(reinterpret_cast<__nv_bfloat162*>(y),
              __halves2bfloat162(__ushort_as_bfloat16(q0), __ushort_as_bfloat16(q1)));
  } else {
    atomicAdd(reinterpret_cast<__half2*>(y), __halves2half2(__ushort_as_half(q0), __ushort_as_half(q1)));
  }
}

template <int RULE>
__device__ __forceinline__ void atomic_add16(uint16_t* y, uint16_t q) {
  if (RULE == kBF16) atomicAdd(reinterpret_cast<__nv_bfloat16*>(y), __ushort_as_bfloat16(q));
  else atomicAdd(reinterpret_cast<__half*>(y), __ushort_as_half(q));
}

// Status word bits written by kernels that detect a problem (never trap).
enum : unsigned { kStatusTimeout = 1u, kStatusNumeric = 2u, kStatusBounds = 4u };

// ------------------------------------------------------------------ mbarrier / TMA (sm_90+ PTX)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive once and add `bytes` to the transaction count the current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Arrive once (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One bounded poll: true once the phase of parity `parity` has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for a phase with an iteration limit; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = (1u << 22)) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Order earlier generic-proxy accesses of shared memory before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 2-D tiled TMA load of one box at (x, y) of `map` into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int32_t x, int32_t y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace sk
