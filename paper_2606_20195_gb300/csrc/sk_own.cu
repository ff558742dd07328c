// Owner kernel: the chunked sketch with exclusive ownership of accumulator rows instead of
// shared-memory atomics.
//
// Paper Sec. 4.1 (scatter of every element of A to its k target rows) with the same chunked FP32
// pre-combine and flush as the tile kernel (sk_tile.cuh). Work item: rows [r0, r1) of chunk t (all
// or a slice), one pair of blocks of S (j0 = 2*bg, kbe = 1 or 2 blocks) and 32 columns [32g, 32g+32).
// The accumulator holds kbe x B x 32 FP32 values in shared memory, line (jl*B + s) per target row.
//
// Ownership: 31 consumer warps alternate over the kbe blocks; each owns a contiguous range of target
// rows of its block. Rows of A arrive through a CTA-wide pipeline of `kOwnDepth` stages of
// kOwnStageRows rows x 32 columns (one TMA box each), run by the 32nd warp: for every stage it
// evaluates the pair's SplitMix64 output of each row, stores its two target words (target row with
// the sign in bit 31) and issues the box. Every consumer warp ballots over the stage's words of its
// block and, for each row
// whose target it owns (in ascending row order), adds the row's 32 values into the target line, one
// lane per column, with a plain shared-memory read-modify-write: no two warps ever touch the same
// line, and the 32 lanes of an access hit 32 consecutive words. Within a work item every
// accumulator value therefore receives its contributions in ascending row order, the canonical FP32
// order; a chunk processed as one work item gives the canonical chunk total exactly.
//
// Pipeline barriers (per stage slot): `full` completes when the producer has stored the target words
// and the TMA box has landed, `empty` when all consumer warps have released the slot. Every wait is
// bounded; on expiry the kernel sets kStatusTimeout, waits (bounded) for its copies in flight and
// leaves.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "sk_internal.h"
#include "sk_tile.cuh"

namespace sk {

namespace {

constexpr int kOwnStageRows = 128;  // rows per stage (TMA box 32 columns x 128 rows = 16 KiB)
constexpr int kOwnDepth = 4;        // stage slots
constexpr int kOwnThreads = 1024;
constexpr int kOwnConsumers = kOwnThreads / 32 - 1;  // warps 0..30 own targets; warp 31 produces

struct OwnSmem {
  size_t acc_off, stage_off, tgt_off, bar_off, total;
};

__host__ __device__ inline OwnSmem own_smem(int64_t acc_floats) {
  OwnSmem L;
  L.acc_off = 0;
  L.stage_off = (((size_t)acc_floats * 4) + 127) & ~(size_t)127;
  L.tgt_off = L.stage_off + (size_t)kOwnDepth * kOwnStageRows * 32 * 4;
  L.bar_off = L.tgt_off + (size_t)kOwnDepth * 2 * kOwnStageRows * 4;
  L.total = L.bar_off + (size_t)2 * kOwnDepth * 8;
  return L;
}

template <int RULE>
__global__ void __launch_bounds__(kOwnThreads, 1) own_kernel(const TileGrid P, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int abort_flag;
  const OwnSmem SL = own_smem(P.acc_floats);
  float* acc = reinterpret_cast<float*>(smem_raw + SL.acc_off);
  float* stages = reinterpret_cast<float*>(smem_raw + SL.stage_off);
  uint32_t* tgt = reinterpret_cast<uint32_t*>(smem_raw + SL.tgt_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + SL.bar_off);
  uint64_t* empty = full + kOwnDepth;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool producer = (warp == kOwnConsumers);
  if (blockDim.x != kOwnThreads || !P.use_tma) {
    if (threadIdx.x == 0 && P.status) atomicOr(P.status, kStatusBounds);
    return;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < kOwnDepth; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, kOwnConsumers);
    }
    mbar_fence_init();
    abort_flag = 0;
  }
  for (int x = threadIdx.x; x < P.acc_floats; x += blockDim.x) acc[x] = 0.f;
  __syncthreads();
  TileDesc D = P.D;
  D.tmap = &tmap;
  const uint32_t B = D.B;
  const int64_t dn = (int64_t)D.B * D.k * D.n;
  const uint32_t box_bytes = (uint32_t)(kOwnStageRows * 32 * 4);
  uint32_t uses = 0;  // stages of this CTA so far (the same count in every warp)
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
    const int32_t nrows = (int32_t)(r1 - r0);
    const int32_t nst = (nrows + kOwnStageRows - 1) / kOwnStageRows;
    bool ok = true;
    if (producer) {
      // Stage s: wait until the consumers released the slot, store the target words of its rows
      // (block j0 and, with two blocks, j0+1: stream output row*kp + j0/2 + 1; with one block per
      // item, j0 & 1 picks the half), then issue its box; the box's arrival completes `full`.
      const int32_t ybase = (int32_t)(r0 - D.row_base);
      const uint32_t pair = (uint32_t)j0 >> 1;
      const bool lo_first = (j0 & 1) != 0;
      int32_t issued = 0;
      for (int32_t s = 0; s < nst; ++s) {
        const uint32_t u = uses + (uint32_t)s;
        const int slot = (int)(u % kOwnDepth);
        if (u >= (uint32_t)kOwnDepth && !mbar_wait_bounded(empty + slot, ((u - kOwnDepth) / kOwnDepth) & 1u)) {
          ok = false;
          break;
        }
        uint32_t* tg = tgt + (size_t)slot * 2 * kOwnStageRows;
#pragma unroll
        for (int q = 0; q < kOwnStageRows / 32; ++q) {
          const int32_t rl = s * kOwnStageRows + q * 32 + lane;  // row of the item
          uint32_t w0 = 0x7FFFFFFFu, w1 = 0x7FFFFFFFu;            // no owner
          if (rl < nrows) {
            const uint64_t h = row_pair_bits(D.seed, (uint64_t)(r0 + rl), D.kp, pair);
            const uint32_t whi = (uint32_t)(h >> 32), wlo = (uint32_t)h;
            const uint32_t wa = lo_first ? wlo : whi;
            w0 = word_to_slot(wa, B) | (wa << 31);
            w1 = word_to_slot(wlo, B) | (wlo << 31);
          }
          tg[q * 32 + lane] = w0;
          if (kbe > 1) tg[kOwnStageRows + q * 32 + lane] = w1;
        }
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(full + slot, box_bytes);
          tma_load_2d(stages + (size_t)slot * kOwnStageRows * 32, D.tmap, g * 32, ybase + s * kOwnStageRows,
                      full + slot);
        }
        issued = s + 1;
      }
      if (!ok && lane == 0) {
        // Leave only after the boxes issued for this item have landed (bounded).
        for (int32_t q = max(0, issued - kOwnDepth); q < issued; ++q) {
          const uint32_t u = uses + (uint32_t)q;
          mbar_wait_bounded(full + (u % kOwnDepth), (u / kOwnDepth) & 1u);
        }
      }
    } else {
      // This warp's block of the pair (warps alternate between the blocks) and its target rows
      // [t_lo, t_lo + tw) of that block.
      const int bw = warp % kbe;
      const int ww = warp / kbe;
      const int wpb = (kOwnConsumers - bw + kbe - 1) / kbe;
      const uint32_t t_lo = (uint32_t)(((uint64_t)ww * B + wpb - 1) / wpb);
      const uint32_t tw = (uint32_t)(((uint64_t)(ww + 1) * B + wpb - 1) / wpb) - t_lo;
      float* accb = acc + (size_t)bw * B * 32 + lane;
      for (int32_t s = 0; s < nst; ++s) {
        const uint32_t u = uses + (uint32_t)s;
        const int slot = (int)(u % kOwnDepth);
        if (!mbar_wait_bounded(full + slot, (u / kOwnDepth) & 1u)) {
          ok = false;
          break;
        }
        const float* st = stages + (size_t)slot * kOwnStageRows * 32 + lane;
        const uint32_t* tg = tgt + (size_t)slot * 2 * kOwnStageRows + bw * kOwnStageRows;
#pragma unroll 1
        for (int grp = 0; grp < kOwnStageRows / 32; ++grp) {
          const uint32_t wv = tg[grp * 32 + lane];
          uint32_t m = __ballot_sync(0xffffffffu, ((wv & 0x7FFFFFFFu) - t_lo) < tw);
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t wb = __shfl_sync(0xffffffffu, wv, b);
            const float a = st[(grp * 32 + b) * 32];
            float* p = accb + (size_t)(wb & 0x7FFFFFFFu) * 32;
            *p += __uint_as_float(__float_as_uint(a) ^ (wb & 0x80000000u));
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
      }
    }
    if (!ok) {
      abort_flag = 1;
      if (P.status) atomicOr(P.status, kStatusTimeout);
    }
    uses += (uint32_t)nst;
    __syncthreads();
    if (abort_flag) break;
    if (P.slices == 1) {
      tile_flush<RULE>(D, t, g, j0, kbe, acc);
    } else {
      // slice partials into the chunk totals; the chunk-finish kernel adds them into Y afterwards
      tile_flush_partial(D, g, j0, kbe, acc, P.P + tl * dn);
    }
    __syncthreads();
  }
}

using OwnKernel = void (*)(const TileGrid, const CUtensorMap);

OwnKernel own_kernel_ptr(int32_t rule) {
  switch (rule) {
    case kRN: return own_kernel<kRN>;
    case kSR: return own_kernel<kSR>;
    case kDither: return own_kernel<kDither>;
    case kBF16: return own_kernel<kBF16>;
    default: return own_kernel<kFP32>;
  }
}

}  // namespace

size_t own_smem_bytes(int64_t B, int32_t kb) { return own_smem((int64_t)kb * B * 32).total; }

int32_t own_threads() { return kOwnThreads; }

int32_t own_ctas_per_sm(int32_t rule, size_t smem) {
  const OwnKernel kern = own_kernel_ptr(rule);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOwnThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

cudaError_t launch_own(const TileLaunch& L, cudaStream_t st, int32_t* launches) {
  // FP32 A only (its staging and consumer loads are written for 4-byte elements)
  if (L.NC != 32 || L.kb < 1 || L.kb > 2 || L.a_type != kAF32) return cudaErrorInvalidValue;
  TileGrid P;
  memset(&P, 0, sizeof(P));
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
  P.D.log2NC = 5;
  P.D.S = 1;
  P.D.kb = L.kb;
  P.D.col_off = L.col_off;
  P.D.tmap = nullptr;
  P.D.mb = 1;
  P.D.lr = 0;
  P.D.vec = 0;
  P.row_begin = L.row_begin;
  P.row_end = L.row_end;
  P.R = L.R;
  P.t_first = L.row_begin / L.R;
  int64_t chunks;
  tile_geometry(L, &chunks, &P.ncg, &P.nbg);
  P.slices = std::max(1, L.slices);
  P.items = chunks * P.slices * P.ncg * P.nbg;
  P.acc_floats = (int32_t)((int64_t)L.kb * B * 32);
  P.P = L.P;
  P.status = L.status;
  P.depth = kOwnDepth;
  if (P.slices > 1 && !P.P) return cudaErrorInvalidValue;
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  if (!encode_a_map(&tmap, L.A, kAF32, L.lda, L.n, L.row_end - L.row_begin, 32, kOwnStageRows))
    return cudaErrorInvalidValue;
  P.use_tma = 1;
  const size_t smem = own_smem((int64_t)P.acc_floats).total;
  const OwnKernel kern = own_kernel_ptr(L.rule);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOwnThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t grid = L.grid > 0 ? L.grid : (int64_t)sms * per_sm;
  grid = std::min<int64_t>(grid, P.items);
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kOwnThreads, smem, st>>>(P, tmap);
  if (launches) *launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (P.slices > 1 && !L.no_finish) return launch_chunk_finish(P.D, L.rule, P.P, P.t_first, chunks, st, launches);
  return cudaSuccess;
}

}  // namespace sk
