// The chunked tile kernel (fast path of the single-matrix sketch), templated on the rounding rule
// and the element type of A. Paper Sec. 4.1 (SparseStack scatter) and Sec. 4.2 (FP16 variants).
#pragma once

#include "sk_tile.cuh"

namespace sk {

// ------------------------------------------------------------------ tile kernel

// One CTA per SM (or per work item), work items in a grid-stride loop: scatter, then flush into Y or
// into the chunk totals. TA is the element type of A; the FP32 instantiations live in sk_kernels.cu,
// the 16-bit ones in sk_kernels_a16.cu (compiled in parallel).
template <int RULE, typename TA>
__global__ void __launch_bounds__(1024) tile_kernel(const TileGrid P, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int abort_flag;
  float* acc = reinterpret_cast<float*>(smem_raw);
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int RBh = 32 / (int)P.D.kp;
  const SmemPlan SL = smem_plan(P.acc_floats, nwarps, ring_slot_bytes(RBh * P.D.mb, 1 << P.D.log2NC), P.depth);
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(smem_raw + SL.wbuf_off) + warp * kWordsPerWarp;
  WarpRing ring = make_ring(smem_raw, SL, warp);
  for (int x = threadIdx.x; x < P.acc_floats; x += blockDim.x) acc[x] = 0.f;
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  TileDesc D = P.D;
  D.tmap = P.use_tma ? (const void*)&tmap : nullptr;
  const int64_t dn = (int64_t)D.B * D.k * D.n;
  for (int64_t w = blockIdx.x; w < P.items; w += gridDim.x) {
    const int32_t g = (int32_t)(w % P.ncg);
    int64_t rest = w / P.ncg;
    const int32_t bg = (int32_t)(rest % P.nbg);
    rest /= P.nbg;
    const int32_t sl = (int32_t)(rest % P.slices);
    const int64_t tl = rest / P.slices;
    const int64_t t = P.t_first + tl;
    const int64_t c0 = max(t * P.R, P.row_begin);
    const int64_t c1 = min((t + 1) * P.R, P.row_end);
    const int64_t r0 = c0 + (c1 - c0) * sl / P.slices;
    const int64_t r1 = c0 + (c1 - c0) * (sl + 1) / P.slices;
    const int32_t j0 = bg * D.kb;
    const int32_t kbe = min(D.kb, (int32_t)D.k - j0);
    if (!tile_scatter_typed<TA>(D, r0, r1, g, j0, kbe, acc, wbuf, ring, warp, nwarps)) {
      abort_flag = 1;
      if (P.status) atomicOr(P.status, kStatusTimeout);
    }
    __syncthreads();
    if (abort_flag) break;
    if (P.slices == 1) {
      tile_flush<RULE>(D, t, g, j0, kbe, acc);
    } else {
      // slice partials into the chunk totals; chunk_finish_kernel adds them into Y after this launch
      tile_flush_partial(D, g, j0, kbe, acc, P.P + tl * dn);
    }
    __syncthreads();
  }
}

using TileKernelFn = void (*)(const TileGrid, const CUtensorMap);

// The tile kernel for a rule and a 16-bit element type of A (kAF16, kABF16), from sk_kernels_a16.cu.
TileKernelFn tile_kernel_a16(int32_t rule, int32_t a_type);

}  // namespace sk
