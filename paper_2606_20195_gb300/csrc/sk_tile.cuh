// One work item of the chunked sketch: rows [r0, r1) of chunk t, columns [g*NC, g*NC + NC) and
// blocks [j0, j0 + kb) of S, accumulated in an FP32 shared-memory tile and then flushed into Y.
//
// Paper Sec. 4.1 (scatter of every element of A to its zeta target rows, Listing 1) and Sec. 4.2
// (FP16 quantization of each contribution, packed half2 atomics, Listing 2). Two changes from the
// paper's per-element design: (1) contributions of the R rows of one chunk that reach the same
// output are first summed in FP32 on chip, and the chunk total is what gets scaled, quantized and
// added into Y; (2) S is never read from memory: its nonzero pattern is regenerated from the
// SplitMix64 stream (one 64-bit output per input row and pair of blocks).
//
// Shared-memory layout of the accumulator: lines of LW = S*NC floats. Block jl of the group (jl in
// [0, kb)) owns lines (jl / S) * B + s for its B target rows s, in slot (jl % S) of width NC.
// A warp is split into G = 32/NC lane groups of NC lanes (one lane per column); in one pass the G
// lane groups handle G (row, block) pairs of the same row batch. When kb >= G and kb % G == 0 the
// G pairs of a pass lie in G different slots, so the 32 lanes touch 32 different banks.
#pragma once

#include "sk_device.cuh"

namespace sk {

struct TileDesc {
  const float* A;   // row 0 of A is global row `row_base`
  void* Y;          // d x n, float or binary16
  int64_t lda;
  int64_t n;
  int64_t row_base;
  uint64_t seed;
  float scale;      // fl32(1/sqrt(k))
  uint32_t B;       // rows per block of S
  uint32_t k;       // blocks (nonzeros per column)
  uint32_t kp;      // ceil(k/2): 64-bit stream outputs per input row
  int32_t log2NC;   // columns per work item = 1 << log2NC (2..5)
  int32_t S;        // slots per accumulator line
  int32_t kb;       // blocks per block group
};

// Floats of the accumulator tile for a descriptor.
__host__ __device__ inline int64_t tile_acc_floats(uint32_t B, int32_t kb, int32_t S, int32_t NC) {
  return (int64_t)((kb + S - 1) / S) * (int64_t)B * (int64_t)S * (int64_t)NC;
}

// Scatter rows [r0, r1) of the work item into the zeroed accumulator `acc`. Called by every warp of
// the CTA; warp `warp` of `nwarps` takes row batches warp, warp + nwarps, ... `hbuf` is this warp's
// 32-entry scratch for the stream outputs of the current batch.
__device__ __forceinline__ void tile_scatter(const TileDesc& D, int64_t r0, int64_t r1, int32_t g, int32_t j0,
                                             int32_t kbe, float* acc, uint64_t* hbuf, int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  const int NC = 1 << D.log2NC;
  const int G = 32 >> D.log2NC;
  const int q = lane >> D.log2NC;
  const int c = lane & (NC - 1);
  const int S = D.S;
  const int LW = S * NC;
  const uint32_t B = D.B;
  const uint32_t kp = D.kp;
  const int64_t col = (int64_t)g * NC + c;
  const bool col_ok = col < D.n;
  const float* __restrict__ Abase = D.A + (col_ok ? col : 0);
  // Rows of one batch: the 32 lanes compute one 64-bit stream output each, kp per row.
  const int RB = 32 / (int)kp;
  const int64_t nrows = r1 - r0;
  const int64_t nbatch = (nrows + RB - 1) / RB;
  // Pair indices p = j/2 of the group span [j0/2, (j0+kbe-1)/2]; batch-local lane L holds
  // (row L / kp, pair L % kp).
  if (kbe >= G) {
    for (int64_t bt = warp; bt < nbatch; bt += nwarps) {
      const int64_t ib = r0 + bt * RB;
      const int nr = (int)min((int64_t)RB, r1 - ib);
      {
        const int rl = lane / (int)kp;
        const int pp = lane - rl * (int)kp;
        hbuf[lane] = (rl < nr) ? row_pair_bits(D.seed, (uint64_t)(ib + rl), kp, (uint32_t)pp) : 0ull;
      }
      __syncwarp();
      for (int rl = 0; rl < nr; ++rl) {
        const int64_t i = ib + rl;
        const float a = col_ok ? __ldg(Abase + (i - D.row_base) * D.lda) : 0.f;
        for (int jb = 0; jb < kbe; jb += G) {
          const int jl = jb + q;
          if (jl < kbe && col_ok) {
            const uint32_t j = (uint32_t)(j0 + jl);
            const uint32_t w = block_word(hbuf[rl * kp + (j >> 1)], j);
            const uint32_t s = word_to_slot(w, B);
            const float v = (w & 1u) ? -a : a;
            atomicAdd(&acc[((jl / S) * (int64_t)B + s) * LW + (jl % S) * NC + c], v);
          }
        }
      }
      __syncwarp();
    }
  } else {
    // Fewer blocks than lane groups: a pass covers RP = G / kbe rows.
    const int RP = G / kbe;
    const int roff = q / kbe;
    const int jl = q - roff * kbe;
    const bool lane_on = roff < RP;
    const uint32_t j = (uint32_t)(j0 + jl);
    for (int64_t bt = warp; bt < nbatch; bt += nwarps) {
      const int64_t ib = r0 + bt * RB;
      const int nr = (int)min((int64_t)RB, r1 - ib);
      {
        const int rl = lane / (int)kp;
        const int pp = lane - rl * (int)kp;
        hbuf[lane] = (rl < nr) ? row_pair_bits(D.seed, (uint64_t)(ib + rl), kp, (uint32_t)pp) : 0ull;
      }
      __syncwarp();
      for (int rb = 0; rb < nr; rb += RP) {
        const int rl = rb + roff;
        if (lane_on && rl < nr && col_ok) {
          const int64_t i = ib + rl;
          const float a = __ldg(Abase + (i - D.row_base) * D.lda);
          const uint32_t w = block_word(hbuf[rl * kp + (j >> 1)], j);
          const uint32_t s = word_to_slot(w, B);
          const float v = (w & 1u) ? -a : a;
          atomicAdd(&acc[((jl / S) * (int64_t)B + s) * LW + (jl % S) * NC + c], v);
        }
      }
      __syncwarp();
    }
  }
}

// Flush the accumulator of a finished work item into Y and zero it. Chunk index t keys the
// rounding random bits. Quads of four consecutive columns are handled together: one Philox call
// gives their four uniforms, FP32 adds use one 16-byte vector reduction, FP16 adds use two packed
// half2 atomics (paper Listing 2). Quads whose four partial sums are all zero are skipped: adding
// a quantized zero leaves Y unchanged.
template <int RULE>
__device__ __forceinline__ void tile_flush(const TileDesc& D, int64_t t, int32_t g, int32_t j0, int32_t kbe,
                                           float* acc) {
  const int NC = 1 << D.log2NC;
  const int S = D.S;
  const int LW = S * NC;
  const uint32_t B = D.B;
  const int nq = NC >> 2;
  const int64_t total = (int64_t)kbe * B * nq;
  const int64_t n = D.n;
  const bool vec4 = (n & 3) == 0;
  const bool even = (n & 1) == 0;
  for (int64_t f = threadIdx.x; f < total; f += blockDim.x) {
    const int c4 = (int)(f % nq);
    const int64_t rest = f / nq;
    const uint32_t s = (uint32_t)(rest % B);
    const int jl = (int)(rest / B);
    float* p = &acc[((jl / S) * (int64_t)B + s) * LW + (jl % S) * NC + 4 * c4];
    float4 v = *reinterpret_cast<float4*>(p);
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
    *reinterpret_cast<float4*>(p) = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t col0 = (int64_t)g * NC + 4 * c4;
    if (col0 >= n) continue;
    const uint32_t r = (uint32_t)(j0 + jl) * B + s;
    const float x0 = __fmul_rn(D.scale, v.x), x1 = __fmul_rn(D.scale, v.y);
    const float x2 = __fmul_rn(D.scale, v.z), x3 = __fmul_rn(D.scale, v.w);
    if (RULE == kFP32) {
      float* y = reinterpret_cast<float*>(D.Y) + (int64_t)r * n + col0;
      if (vec4 && col0 + 3 < n) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(x0), "f"(x1), "f"(x2), "f"(x3)
                     : "memory");
      } else {
        atomicAdd(y, x0);
        if (col0 + 1 < n) atomicAdd(y + 1, x1);
        if (col0 + 2 < n) atomicAdd(y + 2, x2);
        if (col0 + 3 < n) atomicAdd(y + 3, x3);
      }
    } else {
      float u[4] = {0.f, 0.f, 0.f, 0.f};
      if (RULE != kRN) uniforms4(D.seed, r, (uint32_t)(col0 >> 2), (uint64_t)t, u);
      const __half q0 = quantize<RULE>(x0, u[0]);
      const __half q1 = quantize<RULE>(x1, u[1]);
      const __half q2 = quantize<RULE>(x2, u[2]);
      const __half q3 = quantize<RULE>(x3, u[3]);
      __half* y = reinterpret_cast<__half*>(D.Y) + (int64_t)r * n + col0;
      if (even && col0 + 3 < n) {
        atomicAdd(reinterpret_cast<__half2*>(y), __halves2half2(q0, q1));
        atomicAdd(reinterpret_cast<__half2*>(y + 2), __halves2half2(q2, q3));
      } else if (even) {
        atomicAdd(reinterpret_cast<__half2*>(y), __halves2half2(q0, q1));  // col0 + 1 < n since n even
      } else {
        atomicAdd(y, q0);
        if (col0 + 1 < n) atomicAdd(y + 1, q1);
        if (col0 + 2 < n) atomicAdd(y + 2, q2);
        if (col0 + 3 < n) atomicAdd(y + 3, q3);
      }
    }
  }
}

}  // namespace sk
