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

// ------------------------------------------------------------------ global-accumulator kernel
// For blocks too tall for an on-chip accumulator (B x 4 columns of FP32 beyond shared memory): one warp
// per input row (grid-stride over the rows). Lane j < k evaluates block j's word of the row (stream
// output i*kp + j/2 + 1), the lanes then take the row's 4-column quads in turns and add each signed
// quad into the chunk total P[t - t_first][target][...] with one red.global.add.v4.f32 (scalar FP32
// reductions for a ragged last quad or n % 4 != 0). Contributions reach each chunk total in any order
// (atomic mode); chunk_finish_kernel then adds the totals into Y in chunk order.
template <typename TA>
__global__ void __launch_bounds__(256) global_kernel(const TileDesc D, float* P, int64_t row_end, int64_t R,
                                                     int64_t t_first) {
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
      for (int64_t q0 = 0; q0 < nq; q0 += 32) {
        const int64_t q = q0 + lane;
        const bool active = q < nq;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t col0 = 4 * q;
        if (active) {
          if (vec) {
            if constexpr (std::is_same<TA, float>::value) {
              a = __ldg(reinterpret_cast<const float4*>(arow + col0));
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
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w4)
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
  if (L.slices > 1) {
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
      switch (L.a_type) {
        case kAF16: global_kernel<__half><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
        case kABF16: global_kernel<__nv_bfloat16><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
        default: global_kernel<float><<<(unsigned)grid, 256, 0, st>>>(D, L.P, re, L.R, t0); break;
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

cudaError_t launch_tile(const TileLaunch& L, cudaStream_t st, int32_t* launches) {
  if (L.glob) return launch_global(L, st, launches);
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
  if (P.slices > 1) return launch_chunk_finish(P.D, L.rule, P.P, P.t_first, chunks, st, launches);
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
