// The global-accumulator kernel: chunk totals accumulated in device memory with FP32 reductions (one
// warp per input row), for blocks of S too tall for the tile kernel's shared-memory accumulator and
// for the shapes where it is faster (wide matrices at small k, block groups); passes over chunk
// batches and column slabs keep the totals resident in L2. Paper Sec. 4.1 (scatter) and Sec. 4.2
// (the rules, applied by the chunk finish).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "sk_device.cuh"
#include "sk_internal.h"
#include "sk_tile.cuh"

namespace sk {

// L2 eviction priorities: rows of A are read once (evict first), the chunk totals are reduced into
// again and again while A streams past (evict last), so A's lines are the ones the L2 gives up.
__device__ __forceinline__ uint64_t pol_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t pol_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_first(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
  return v;
}

// ------------------------------------------------------------------ global-accumulator kernel
// For blocks too tall for an on-chip accumulator (B x 4 columns of FP32 beyond shared memory): one warp
// per input row (grid-stride over the rows). Lane j < k evaluates block j's word of the row (stream
// output i*kp + j/2 + 1), the lanes then take the row's 4-column quads in turns and add each signed
// quad into the chunk total P[t - t_first][target][...] with one red.global.add.v4.f32 (scalar FP32
// reductions for a ragged last quad or n % 4 != 0). Contributions reach each chunk total in any order
// (atomic mode); chunk_finish_kernel then adds the totals into Y in chunk order.
template <typename TA, int QB>
__global__ void __launch_bounds__(256) global_kernel(const TileDesc D, float* P, int64_t row_end, int64_t R,
                                                     int64_t t_first) {
  const uint64_t pf = pol_first(), pl = pol_last();
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = D.n;
  const int64_t nq = (n + 3) >> 2;
  const int k = (int)D.k;
  const int64_t dn = (int64_t)D.B * D.k * n;
  // quads of A in one vector load: 16 bytes of FP32 or 8 bytes of 16-bit values
  const bool vec = (n & 3) == 0 && (D.lda & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(D.A) & (std::is_same<TA, float>::value ? 15u : 7u)) == 0;
  for (int64_t i = D.row_base + wg; i < row_end; i += nw) {
    float* Pt = P + (i / R - t_first) * dn;
    const TA* arow = static_cast<const TA*>(D.A) + (i - D.row_base) * D.lda;
    for (int jb = 0; jb < k; jb += 32) {
      // this lane's block jb + lane: target row (with the block offset) and sign bit
      uint32_t tw = 0;
      const int jl = jb + lane;
      if (jl < k) {
        const uint32_t w = block_word(row_pair_bits(D.seed, (uint64_t)i, D.kp, (uint32_t)jl >> 1), (uint32_t)jl);
        tw = ((uint32_t)jl * D.B + word_to_slot(w, D.B)) | (w << 31);
      }
      const int kk = min(32, k - jb);
      if constexpr (QB == 1) {
        for (int64_t q0 = 0; q0 < nq; q0 += 32) {
          const int64_t q = q0 + lane;
          const bool active = q < nq;
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
          const int64_t col0 = 4 * q;
          if (active) {
            if (vec) {
              if constexpr (std::is_same<TA, float>::value) {
                a = ld_first(reinterpret_cast<const float4*>(arow + col0), pf);
              } else {
                const uint2 u = __ldg(reinterpret_cast<const uint2*>(arow + col0));
                const TA* h = reinterpret_cast<const TA*>(&u);
                a = make_float4(a_to_f32(h[0]), a_to_f32(h[1]), a_to_f32(h[2]), a_to_f32(h[3]));
              }
            } else {
              a.x = ld_a(arow + col0);
              if (col0 + 1 < n) a.y = ld_a(arow + col0 + 1);
              if (col0 + 2 < n) a.z = ld_a(arow + col0 + 2);
              if (col0 + 3 < n) a.w = ld_a(arow + col0 + 3);
            }
          }
          for (int jj = 0; jj < kk; ++jj) {
            const uint32_t t = __shfl_sync(0xffffffffu, tw, jj);
            if (!active) continue;
            const uint32_t sg = t & 0x80000000u;
            float* p = Pt + (int64_t)(t & 0x7FFFFFFFu) * n + col0;
            const float x = __uint_as_float(__float_as_uint(a.x) ^ sg), y = __uint_as_float(__float_as_uint(a.y) ^ sg);
            const float z = __uint_as_float(__float_as_uint(a.z) ^ sg), w4 = __uint_as_float(__float_as_uint(a.w) ^ sg);
            if ((n & 3) == 0) {
              asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w4), "l"(pl)
                           : "memory");
            } else {
              atomicAdd(p, x);
              if (col0 + 1 < n) atomicAdd(p + 1, y);
              if (col0 + 2 < n) atomicAdd(p + 2, z);
              if (col0 + 3 < n) atomicAdd(p + 3, w4);
            }
          }
        }
      } else {
        // QB quads per lane are loaded before any of their reductions, so that a warp has QB row
        // loads in flight (the reductions' memory clobber keeps later loads from moving above them).
        for (int64_t q0 = 0; q0 < nq; q0 += 32 * QB) {
          float4 a[QB];
#pragma unroll
          for (int b = 0; b < QB; ++b) {
            const int64_t q = q0 + b * 32 + lane;
            a[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q >= nq) continue;
            const int64_t col0 = 4 * q;
            if (vec) {
              if constexpr (std::is_same<TA, float>::value) {
                a[b] = ld_first(reinterpret_cast<const float4*>(arow + col0), pf);
              } else {
                const uint2 u = __ldg(reinterpret_cast<const uint2*>(arow + col0));
                const TA* h = reinterpret_cast<const TA*>(&u);
                a[b] = make_float4(a_to_f32(h[0]), a_to_f32(h[1]), a_to_f32(h[2]), a_to_f32(h[3]));
              }
            } else {
              a[b].x = ld_a(arow + col0);
              if (col0 + 1 < n) a[b].y = ld_a(arow + col0 + 1);
              if (col0 + 2 < n) a[b].z = ld_a(arow + col0 + 2);
              if (col0 + 3 < n) a[b].w = ld_a(arow + col0 + 3);
            }
          }
          for (int jj = 0; jj < kk; ++jj) {
            const uint32_t t = __shfl_sync(0xffffffffu, tw, jj);
            const uint32_t sg = t & 0x80000000u;
            float* prow = Pt + (int64_t)(t & 0x7FFFFFFFu) * n;
#pragma unroll
            for (int b = 0; b < QB; ++b) {
              const int64_t q = q0 + b * 32 + lane;
              if (q >= nq) break;
              const int64_t col0 = 4 * q;
              float* p = prow + col0;
              const float x = __uint_as_float(__float_as_uint(a[b].x) ^ sg);
              const float y = __uint_as_float(__float_as_uint(a[b].y) ^ sg);
              const float z = __uint_as_float(__float_as_uint(a[b].z) ^ sg);
              const float w4 = __uint_as_float(__float_as_uint(a[b].w) ^ sg);
              if ((n & 3) == 0) {
                asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w4), "l"(pl)
                             : "memory");
              } else {
                atomicAdd(p, x);
                if (col0 + 1 < n) atomicAdd(p + 1, y);
                if (col0 + 2 < n) atomicAdd(p + 2, z);
                if (col0 + 3 < n) atomicAdd(p + 3, w4);
              }
            }
          }
        }
      }
    }
  }
}

// Chunk totals of one pass kept at most this large, so that they stay in L2 (129 MB) while A streams
// past: beyond it the FP32 reductions into P miss L2 and each total line travels to DRAM and back
// several times.
constexpr int64_t kGlobalPassBytes = (int64_t)40 << 20;

// Measured on GB300 (n = 1024, m = 2^21): with k = 4, passes raise the throughput at d/n = 16, 32 and
// 64 by 28-46 %; slabs narrower than 128 columns leave most lanes of a row's warp idle and repeat the
// row's hash per slab (d/n = 256: 622 -> 368 GB/s), and at k = 1 (few reductions per row) the extra
// launches cost more than the L2 misses they avoid. Those cases keep one pass over all chunks.
void global_passes(const TileLaunch& L, int64_t* ns, int64_t* cb) {
  const int64_t t_first = L.row_begin / L.R;
  const int64_t chunks = (L.row_end - 1) / L.R - t_first + 1;
  const int64_t per_col = L.d * 4;  // bytes of one column of one chunk total
  *ns = L.n;
  *cb = chunks;
  if (chunks * L.n * per_col <= kGlobalPassBytes || L.k < 2) return;
  const int64_t cb_fit = kGlobalPassBytes / (L.n * per_col);
  if (cb_fit >= 1) {
    *cb = cb_fit;
    return;
  }
  // one chunk at a time is still too large: column slabs (multiples of 4 columns), if wide enough
  const int64_t slab = (kGlobalPassBytes / per_col) & ~(int64_t)3;
  if (slab < 128) return;
  *cb = 1;
  *ns = slab;
}

int64_t launch_P_floats(const TileLaunch& L) {
  if (L.glob) {
    int64_t ns, cb;
    global_passes(L, &ns, &cb);
    return cb * L.d * ns;
  }
  if (L.slices > 1 || L.reg) {
    int64_t chunks;
    int32_t ncg, nbg;
    tile_geometry(L, &chunks, &ncg, &nbg);
    return chunks * L.d * L.n;
  }
  return 0;
}

// The global-accumulator kernel in passes (column slabs x chunk batches, ascending chunks within
// each slab): each pass reduces into P and its chunk finish adds the pass's chunk totals into Y in
// chunk order and clears P for the next pass.
cudaError_t launch_global(const TileLaunch& L, cudaStream_t st, int32_t* launches) {
  if (!L.P) return cudaErrorInvalidValue;
  const int64_t B = L.d / L.k;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t ns, cb;
  global_passes(L, &ns, &cb);
  const size_t es_a = (L.a_type == kAF32) ? 4 : 2;
  const size_t es_y = (L.rule == kFP32) ? 4 : 2;
  const int64_t t_begin = L.row_begin / L.R;
  const int64_t t_end = (L.row_end - 1) / L.R;
  // Four quads of a row per lane in flight on wide rows (measured on GB300 at n = 256 and 1024: +5 to
  // +13 %; at n = 64 the lanes of a row's warp are mostly idle and the larger register count costs
  // 20 %); at k = 1 with chunk totals beyond L2 the extra loads compete with the L2-missing
  // reductions (-5 to -10 %), so one quad per lane there.
  const bool qb4 = ns >= 256 && !(L.k == 1 && cb * L.d * ns * 4 > ((int64_t)128 << 20));
  for (int64_t c0 = 0; c0 < L.n; c0 += ns) {
    const int64_t nsl = std::min(ns, L.n - c0);
    for (int64_t t0 = t_begin; t0 <= t_end; t0 += cb) {
      const int64_t t1 = std::min(t0 + cb - 1, t_end);
      const int64_t rb = std::max(L.row_begin, t0 * L.R);
      const int64_t re = std::min(L.row_end, (t1 + 1) * L.R);
      TileDesc D;
      memset(&D, 0, sizeof(D));
      D.A = static_cast<const char*>(L.A) + es_a * (size_t)((rb - L.row_begin) * L.lda + c0);
      D.a_type = L.a_type;
      D.Y = static_cast<char*>(L.Y) + es_y * (size_t)c0;
      D.ldy = L.n;
      D.lda = L.lda;
      D.n = nsl;
      D.row_base = rb;
      D.seed = L.seed;
      D.scale = L.scale;
      D.B = (uint32_t)B;
      D.k = (uint32_t)L.k;
      D.kp = (uint32_t)((L.k + 1) / 2);
      D.log2NC = 2;
      D.S = 1;
      D.kb = L.k;
      D.col_off = L.col_off + c0;
      const int64_t rows = re - rb;
      const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)sms * 8));
      if (qb4) {
        switch (L.a_type) {
          case kAF16: global_kernel<__half, 4><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
          case kABF16: global_kernel<__nv_bfloat16, 4><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
          default: global_kernel<float, 4><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
        }
      } else {
        switch (L.a_type) {
          case kAF16: global_kernel<__half, 1><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
          case kABF16: global_kernel<__nv_bfloat16, 1><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
          default: global_kernel<float, 1><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
        }
      }
      if (launches) *launches += 1;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      e = launch_chunk_finish(D, L.rule, L.P, t0, t1 - t0 + 1, st, launches);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace sk
