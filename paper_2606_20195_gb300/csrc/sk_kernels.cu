// Single-matrix sketch kernels: the chunked tile kernel (fast path), the paper-literal per-element
// kernel (comparator), the canonical-order deterministic kernel (verification), and the S pattern
// kernel. Paper Sec. 4.1 (SparseStack scatter) and Sec. 4.2 (FP16 variants).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "sk_device.cuh"
#include "sk_internal.h"
#include "sk_tile.cuh"
#include "sk_tile_kernel.cuh"

namespace sk {

static TileKernelFn tile_kernel_f32(int32_t rule) {
  switch (rule) {
    case kRN: return tile_kernel<kRN, float>;
    case kSR: return tile_kernel<kSR, float>;
    case kDither: return tile_kernel<kDither, float>;
    case kBF16: return tile_kernel<kBF16, float>;
    default: return tile_kernel<kFP32, float>;
  }
}

int32_t tile_slots(int32_t NC, int32_t kb) { return std::min(32 / NC, kb); }

size_t tile_smem_bytes(int64_t B, int32_t kb, int32_t NC, int32_t threads, int32_t k, int32_t depth, int32_t mb) {
  const int32_t S = tile_slots(NC, kb);
  const int64_t fl = tile_acc_floats((uint32_t)B, kb, S, NC);
  const int32_t RB = 32 / ((k + 1) / 2);
  return smem_plan(fl, threads / 32, ring_slot_bytes(RB * mb, NC), depth).total;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

bool encode_a_map(void* map, const void* A, int32_t a_type, int64_t lda, int64_t n, int64_t rows, int32_t NC,
                  int32_t RB) {
  const int64_t es = (a_type == kAF32) ? 4 : 2;
  // 16-byte-aligned base, row stride and box width (the box width rule: NC * es a multiple of 16)
  if ((reinterpret_cast<uintptr_t>(A) & 15u) != 0 || (lda * es) % 16 != 0 || ((int64_t)NC * es) % 16 != 0 ||
      rows >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) || RB > 256 || NC > 256)
    return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(lda * es)};
  const cuuint32_t box[2] = {(cuuint32_t)NC, (cuuint32_t)RB};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = (a_type == kAF16)    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : (a_type == kABF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), dt, 2, (void*)A, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

void tile_geometry(const TileLaunch& L, int64_t* chunks, int32_t* ncg, int32_t* nbg) {
  const int64_t t_first = L.row_begin / L.R;
  const int64_t t_last = (L.row_end - 1) / L.R;
  *chunks = t_last - t_first + 1;
  *ncg = (int32_t)((L.n + L.NC - 1) / L.NC);
  *nbg = (L.k + L.kb - 1) / L.kb;
}

cudaError_t launch_tile(const TileLaunch& L, cudaStream_t st, int32_t* launches) {
  if (L.glob) return launch_global(L, st, launches);
  if (L.reg) return launch_reg(L, st, launches);
  if (L.own) return launch_own(L, st, launches);
  TileGrid P;
  const int64_t B = L.d / L.k;
  P.D.A = L.A;
  P.D.Y = L.Y;
  P.D.lda = L.lda;
  P.D.n = L.n;
  P.D.row_base = L.row_begin;
  P.D.seed = L.seed;
  P.D.scale = L.scale;
  P.D.B = (uint32_t)B;
  P.D.k = (uint32_t)L.k;
  P.D.kp = (uint32_t)((L.k + 1) / 2);
  P.D.log2NC = ilog2(L.NC);
  P.D.S = tile_slots(L.NC, L.kb);
  P.D.kb = L.kb;
  P.row_begin = L.row_begin;
  P.row_end = L.row_end;
  P.R = L.R;
  P.t_first = L.row_begin / L.R;
  int64_t chunks;
  tile_geometry(L, &chunks, &P.ncg, &P.nbg);
  P.slices = std::max(1, L.slices);
  P.items = chunks * P.slices * P.ncg * P.nbg;
  P.acc_floats = (int32_t)tile_acc_floats((uint32_t)B, L.kb, P.D.S, L.NC);
  P.P = L.P;
  P.status = L.status;
  P.D.col_off = L.col_off;
  P.D.a_type = L.a_type;
  P.D.ldy = 0;
  P.D.tmap = nullptr;
  if (P.slices > 1 && !P.P) return cudaErrorInvalidValue;
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  const int32_t RB = 32 / (int32_t)P.D.kp;
  P.D.mb = std::max(1, L.mb);
  P.use_tma = (L.allow_tma &&
                encode_a_map(&tmap, L.A, L.a_type, L.lda, L.n, L.row_end - L.row_begin, L.NC, RB * P.D.mb)) ? 1 : 0;
  P.D.lr = (P.use_tma && L.lr && L.kb == L.k) ? 1 : 0;
  P.D.vec = (L.vec && L.n == 1 && L.NC == 4) ? 1 : 0;
  if (P.D.vec) {
    P.use_tma = 0;
    P.D.lr = 0;
  }
  P.depth = std::max(1, L.depth);
  const size_t smem = tile_smem_bytes(B, L.kb, L.NC, L.threads, L.k, P.depth, P.D.mb);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const TileKernelFn kern = (L.a_type == kAF32) ? tile_kernel_f32(L.rule) : tile_kernel_a16(L.rule, L.a_type);
  if (!kern) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = L.grid > 0 ? L.grid : (int64_t)sms * per_sm;
  grid = std::min<int64_t>(grid, P.items);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, L.threads, smem, st>>>(P, tmap);
  if (launches) *launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (P.slices > 1 && !L.no_finish) return launch_chunk_finish(P.D, L.rule, P.P, P.t_first, chunks, st, launches);
  return cudaSuccess;
}

// ------------------------------------------------------------------ chunk finish
// One thread per output quad (row, 4 columns): the chunks of the launch in ascending order (finish_quad).
template <int RULE>
__global__ void __launch_bounds__(256) chunk_finish_kernel(const TileDesc D, float* P, int64_t t_first, int64_t chunks) {
  const int64_t nq = (D.n + 3) >> 2;
  const int64_t d = (int64_t)D.B * D.k;
  const int64_t dn = d * D.n;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < d * nq; f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = f / nq;
    finish_quad<RULE>(D, (uint32_t)r, 4 * (f - r * nq), P, t_first, chunks, dn);
  }
}

cudaError_t launch_chunk_finish(const TileDesc& D, int32_t rule, float* P, int64_t t_first, int64_t chunks,
                                cudaStream_t st, int32_t* launches) {
  const int64_t quads = (int64_t)D.B * D.k * ((D.n + 3) >> 2);
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((quads + 255) / 256, 1 << 16));
  switch (rule) {
    case kRN: chunk_finish_kernel<kRN><<<grid, 256, 0, st>>>(D, P, t_first, chunks); break;
    case kSR: chunk_finish_kernel<kSR><<<grid, 256, 0, st>>>(D, P, t_first, chunks); break;
    case kDither: chunk_finish_kernel<kDither><<<grid, 256, 0, st>>>(D, P, t_first, chunks); break;
    case kBF16: chunk_finish_kernel<kBF16><<<grid, 256, 0, st>>>(D, P, t_first, chunks); break;
    default: chunk_finish_kernel<kFP32><<<grid, 256, 0, st>>>(D, P, t_first, chunks); break;
  }
  if (launches) *launches += 1;
  return cudaGetLastError();
}

int32_t tile_ctas_per_sm(int32_t rule, int32_t threads, size_t smem) {
  const TileKernelFn kern = tile_kernel_f32(rule);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

// ------------------------------------------------------------------ paper-literal kernel
// One thread per (input row, column pair): for each of the k nonzeros of the row's column of S,
// scale, quantize (FP16 rules) and add with one atomic per element (FP32) or one packed half2
// atomic per column pair (paper Listings 1 and 2). Equivalent to chunk length R = 1; the rounding
// bits of contribution i use chunk index t = i.
template <int RULE>
__global__ void literal_kernel(const LiteralLaunch L, uint32_t B, uint32_t kp) {
  const int64_t n = L.n;
  const int64_t ncp = (n + 1) >> 1;
  const int64_t total = (L.row_end - L.row_begin) * ncp;
  const bool even = (n & 1) == 0;
  for (int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tid < total;
       tid += (int64_t)gridDim.x * blockDim.x) {
    const int64_t il = tid / ncp;
    const int64_t c0 = 2 * (tid - il * ncp);
    const int64_t i = L.row_begin + il;
    const bool has1 = c0 + 1 < n;
    const float a0 = ld_a_any(L.A, L.a_type, il * L.lda + c0);
    const float a1 = has1 ? ld_a_any(L.A, L.a_type, il * L.lda + c0 + 1) : 0.f;
    uint64_t bits = 0;
    for (uint32_t j = 0; j < (uint32_t)L.k; ++j) {
      if ((j & 1u) == 0) bits = row_pair_bits(L.seed, (uint64_t)i, kp, j >> 1);
      const uint32_t w = block_word(bits, j);
      const uint32_t r = j * B + word_to_slot(w, B);
      const bool neg = (w & 1u) != 0;
      const float x0 = __fmul_rn(L.scale, neg ? -a0 : a0);
      const float x1 = __fmul_rn(L.scale, neg ? -a1 : a1);
      if (RULE == kFP32) {
        float* y = reinterpret_cast<float*>(L.Y) + (int64_t)r * n + c0;
        atomicAdd(y, x0);
        if (has1) atomicAdd(y + 1, x1);
      } else {
        float u[4] = {0.f, 0.f, 0.f, 0.f}, u1n[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t cg = L.col_off + c0;
        if (rule_draws_bits<RULE>()) {
          uniforms4(L.seed, r, (uint32_t)(cg >> 2), (uint64_t)i, u);
          if ((cg & 3) == 3 && has1) uniforms4(L.seed, r, (uint32_t)(cg >> 2) + 1u, (uint64_t)i, u1n);
        }
        const uint16_t q0 = quantize16<RULE>(x0, u[cg & 3]);
        uint16_t* y = reinterpret_cast<uint16_t*>(L.Y) + (int64_t)r * n + c0;
        if (has1) {
          const uint16_t q1 = quantize16<RULE>(x1, ((cg & 3) == 3) ? u1n[0] : u[(cg + 1) & 3]);
          if (even) {
            atomic_add16x2<RULE>(y, q0, q1);
          } else {
            atomic_add16<RULE>(y, q0);
            atomic_add16<RULE>(y + 1, q1);
          }
        } else {
          atomic_add16<RULE>(y, q0);
        }
      }
    }
  }
}

cudaError_t launch_literal(const LiteralLaunch& L, cudaStream_t st, int32_t* launches) {
  const uint32_t B = (uint32_t)(L.d / L.k);
  const uint32_t kp = (uint32_t)((L.k + 1) / 2);
  const int64_t total = (L.row_end - L.row_begin) * ((L.n + 1) / 2);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  int64_t grid = std::min<int64_t>((total + threads - 1) / threads, (int64_t)sms * 8);
  if (grid < 1) grid = 1;
  switch (L.rule) {
    case kRN: literal_kernel<kRN><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kSR: literal_kernel<kSR><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kDither: literal_kernel<kDither><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kBF16: literal_kernel<kBF16><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    default: literal_kernel<kFP32><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
  }
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ deterministic kernel
// Canonical order, bit for bit: one thread owns (block j, column c), i.e. outputs (jB..jB+B-1, c).
// For every chunk it sums sign * A[i, c] over ascending rows into the FP32 partials P[s, c]
// (from +0), then walks the chunk's rows again: at the first visit of a target the chunk total is
// scaled, quantized and added into Y in FP32 or binary16 (round to nearest even), and the partial
// is reset to +0; later visits of the same target add a quantized +0, which leaves Y unchanged.
template <int RULE>
__global__ void det_kernel(const DetLaunch L, uint32_t B, uint32_t kp) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n;
  if (tid >= (int64_t)L.k * n) return;
  const uint32_t j = (uint32_t)(tid / n);
  const int64_t c = tid - (int64_t)j * n;
  const int64_t t0 = L.row_begin / L.R;
  const int64_t t1 = (L.row_end - 1) / L.R;
  for (int64_t t = t0; t <= t1; ++t) {
    const int64_t r0 = max(t * L.R, L.row_begin);
    const int64_t r1 = min((t + 1) * L.R, L.row_end);
    for (int64_t i = r0; i < r1; ++i) {
      const uint32_t w = block_word(row_pair_bits(L.seed, (uint64_t)i, kp, j >> 1), j);
      const int64_t r = (int64_t)j * B + word_to_slot(w, B);
      const float a = ld_a_any(L.A, L.a_type, (i - L.row_begin) * L.lda + c);
      float* p = L.P + r * n + c;
      *p = __fadd_rn(*p, (w & 1u) ? -a : a);
    }
    for (int64_t i = r0; i < r1; ++i) {
      const uint32_t w = block_word(row_pair_bits(L.seed, (uint64_t)i, kp, j >> 1), j);
      const int64_t r = (int64_t)j * B + word_to_slot(w, B);
      float* p = L.P + r * n + c;
      const float x = __fmul_rn(L.scale, *p);
      *p = 0.f;
      if (RULE == kFP32) {
        float* y = reinterpret_cast<float*>(L.Y) + r * n + c;
        *y = __fadd_rn(*y, x);
      } else {
        float u[4] = {0.f, 0.f, 0.f, 0.f};
        const int64_t cg = L.col_off + c;
        if (rule_draws_bits<RULE>()) uniforms4(L.seed, (uint32_t)r, (uint32_t)(cg >> 2), (uint64_t)t, u);
        uint16_t* y = reinterpret_cast<uint16_t*>(L.Y) + r * n + c;
        *y = add16<RULE>(*y, quantize16<RULE>(x, u[cg & 3]));
      }
    }
  }
}

cudaError_t launch_det(const DetLaunch& L, cudaStream_t st, int32_t* launches) {
  const uint32_t B = (uint32_t)(L.d / L.k);
  const uint32_t kp = (uint32_t)((L.k + 1) / 2);
  cudaError_t e = cudaMemsetAsync(L.P, 0, sizeof(float) * (size_t)(L.d * L.n), st);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)L.k * L.n;
  const int threads = 128;
  const int64_t grid = (total + threads - 1) / threads;
  switch (L.rule) {
    case kRN: det_kernel<kRN><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kSR: det_kernel<kSR><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kDither: det_kernel<kDither><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    case kBF16: det_kernel<kBF16><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
    default: det_kernel<kFP32><<<(unsigned)grid, threads, 0, st>>>(L, B, kp); break;
  }
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ S pattern
__global__ void pattern_kernel(int64_t d, int32_t k, uint64_t seed, int64_t i0, int64_t cnt, int32_t* rows,
                               int8_t* signs) {
  const uint32_t B = (uint32_t)(d / k);
  const uint32_t kp = (uint32_t)((k + 1) / 2);
  const int64_t total = cnt * k;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = x / k;
    const uint32_t j = (uint32_t)(x - q * k);
    const uint32_t w = block_word(row_pair_bits(seed, (uint64_t)(i0 + q), kp, j >> 1), j);
    rows[x] = (int32_t)(j * B + word_to_slot(w, B));
    signs[x] = (w & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_pattern(int64_t d, int32_t k, uint64_t seed, int64_t i0, int64_t cnt, int32_t* rows,
                           int8_t* signs, cudaStream_t st) {
  const int64_t total = cnt * k;
  const int threads = 256;
  int64_t grid = std::min<int64_t>((total + threads - 1) / threads, 65535);
  if (grid < 1) grid = 1;
  pattern_kernel<<<(unsigned)grid, threads, 0, st>>>(d, k, seed, i0, cnt, rows, signs);
  return cudaGetLastError();
}

}  // namespace sk
