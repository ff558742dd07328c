// Batched uneven sketches in one persistent launch. Every matrix of the batch is cut into work
// items (chunk of rows x column group x block group), the items of all matrices are sorted by cost
// (largest first) into one device work list, and resident CTAs take items from it through an atomic
// counter until it is exhausted. The per-item processing is the tile scatter/flush of the
// single-matrix kernel (paper Sec. 4.1-4.2 with on-chip chunk accumulation).
//
// sk_batch_launch enqueues exactly two kernels (zero every Y_i and reset the counter; then the
// persistent kernel), allocates nothing and never synchronizes, so it can be captured in a CUDA
// graph and replayed.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sk.h"
#include "sk_device.cuh"
#include "sk_hostutil.h"
#include "sk_internal.h"
#include "sk_tile.cuh"

namespace sk {

struct BatchDesc {
  TileDesc D;
  int64_t R;
};

struct BatchWork {
  int64_t r0, r1, t;
  int32_t item, g, j0, kbe;
};

struct ZeroSpan {
  void* p;
  int64_t bytes;
};

__global__ void batch_zero_kernel(const ZeroSpan* spans, int32_t nspan, int32_t* counter) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  for (int32_t s = blockIdx.y; s < nspan; s += gridDim.y) {
    const ZeroSpan z = spans[s];
    // spans are 4-byte aligned and sized (d x n floats or d x n halves padded to 4 bytes)
    uint32_t* p = reinterpret_cast<uint32_t*>(z.p);
    const int64_t words = z.bytes >> 2;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < words; x += (int64_t)gridDim.x * blockDim.x)
      p[x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (z.bytes & 3)) {
      reinterpret_cast<uint16_t*>(z.p)[(z.bytes >> 1) - 1] = 0;
    }
  }
}

template <int RULE>
__global__ void __launch_bounds__(1024) batch_kernel(const BatchDesc* __restrict__ descs,
                                                     const BatchWork* __restrict__ work, int64_t nwork,
                                                     int32_t* counter, int64_t acc_floats, int32_t slot_bytes,
                                                     int32_t depth, unsigned* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int64_t next;
  __shared__ BatchDesc dsh;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  float* acc = reinterpret_cast<float*>(smem_raw);
  const SmemPlan SL = smem_plan(acc_floats, nwarps, slot_bytes, depth);
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(smem_raw + SL.wbuf_off) + warp * kWordsPerWarp;
  WarpRing ring = make_ring(smem_raw, SL, warp);
  for (int64_t x = threadIdx.x; x < acc_floats; x += blockDim.x) acc[x] = 0.f;
  if (threadIdx.x == 0) abort_flag = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) next = (int64_t)atomicAdd(counter, 1);
    __syncthreads();
    const int64_t w = next;
    if (w >= nwork || abort_flag) break;
    const BatchWork wk = work[w];
    if (threadIdx.x == 0) dsh = descs[wk.item];
    __syncthreads();
    if (!tile_scatter_typed<float>(dsh.D, wk.r0, wk.r1, wk.g, wk.j0, wk.kbe, acc, wbuf, ring, warp, nwarps)) {
      abort_flag = 1;
      if (status) atomicOr(status, kStatusTimeout);
    }
    __syncthreads();
    if (abort_flag) break;
    tile_flush<RULE>(dsh.D, wk.t, wk.g, wk.j0, wk.kbe, acc);
    __threadfence();
    __syncthreads();
  }
}

static const void* batch_kernel_ptr(int rule) {
  switch (rule) {
    case kRN: return (const void*)batch_kernel<kRN>;
    case kSR: return (const void*)batch_kernel<kSR>;
    case kDither: return (const void*)batch_kernel<kDither>;
    case kBF16: return (const void*)batch_kernel<kBF16>;
    default: return (const void*)batch_kernel<kFP32>;
  }
}

cudaError_t launch_batch(const void* descs, const void* work, int64_t nwork, int32_t* counter, const void* zero_list,
                         int32_t nzero, int32_t rule, int32_t threads, size_t smem, int32_t grid, int64_t acc_floats,
                         int32_t slot_bytes, int32_t depth, unsigned* status, cudaStream_t st, int32_t* launches) {
  dim3 zg(64, (unsigned)std::min(nzero, 1024));
  batch_zero_kernel<<<zg, 256, 0, st>>>(reinterpret_cast<const ZeroSpan*>(zero_list), nzero, counter);
  if (launches) *launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const BatchDesc* dd = reinterpret_cast<const BatchDesc*>(descs);
  const BatchWork* ww = reinterpret_cast<const BatchWork*>(work);
  // The dynamic shared-memory limit is per-kernel state that another batch may have lowered.
  e = cudaFuncSetAttribute(batch_kernel_ptr(rule), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  switch (rule) {
    case kRN: batch_kernel<kRN><<<grid, threads, smem, st>>>(dd, ww, nwork, counter, acc_floats, slot_bytes, depth, status); break;
    case kSR: batch_kernel<kSR><<<grid, threads, smem, st>>>(dd, ww, nwork, counter, acc_floats, slot_bytes, depth, status); break;
    case kDither: batch_kernel<kDither><<<grid, threads, smem, st>>>(dd, ww, nwork, counter, acc_floats, slot_bytes, depth, status); break;
    case kBF16: batch_kernel<kBF16><<<grid, threads, smem, st>>>(dd, ww, nwork, counter, acc_floats, slot_bytes, depth, status); break;
    default: batch_kernel<kFP32><<<grid, threads, smem, st>>>(dd, ww, nwork, counter, acc_floats, slot_bytes, depth, status); break;
  }
  if (launches) *launches += 1;
  return cudaGetLastError();
}

}  // namespace sk

using namespace sk;

struct sk_batch_s {
  std::vector<sk_batch_item> items;
  int32_t rule = 0;
  int32_t threads = 0, tile_cols = 0;
  int64_t chunk_rows = 0;
  int64_t item_chunks = 0;  // > 0: each item's chunk length from its own m (SK_PARAM_ITEM_CHUNKS)
  bool built = false;
  int device = 0;
  // device state
  CUtensorMap* d_maps = nullptr;
  unsigned* d_status = nullptr;
  int64_t acc_floats = 0;
  int32_t slot_bytes = 0;
  int32_t depth = 1;
  BatchDesc* d_descs = nullptr;
  BatchWork* d_work = nullptr;
  ZeroSpan* d_zero = nullptr;
  int32_t* d_counter = nullptr;
  int64_t nwork = 0;
  int64_t bytes_A = 0;
  size_t smem = 0;
  int32_t grid = 0, use_threads = 0;
  // Device buffers are grown, never shrunk, so a batch rebound to new items reuses them; the host
  // copies of the uploaded tables stay alive until the asynchronous uploads have run.
  size_t cap_maps = 0, cap_descs = 0, cap_work = 0, cap_zero = 0;
  std::vector<CUtensorMap> h_maps;
  std::vector<BatchDesc> h_descs;
  std::vector<BatchWork> h_work;
  std::vector<ZeroSpan> h_zero;
};

namespace {

void free_batch_dev(sk_batch_s* b) {
  if (b->d_maps) cudaFree(b->d_maps);
  if (b->d_status) cudaFree(b->d_status);
  b->d_maps = nullptr;
  b->d_status = nullptr;
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_work) cudaFree(b->d_work);
  if (b->d_zero) cudaFree(b->d_zero);
  if (b->d_counter) cudaFree(b->d_counter);
  b->d_descs = nullptr;
  b->d_work = nullptr;
  b->d_zero = nullptr;
  b->d_counter = nullptr;
  b->cap_maps = b->cap_descs = b->cap_work = b->cap_zero = 0;
}

// Device array of at least `count` elements of T in *ptr (capacity *cap, in elements): kept if large
// enough, else replaced (grown to 1.5x, so a batch rebound to slowly growing item lists reallocates
// rarely).
template <typename T>
bool ensure_dev(T** ptr, size_t* cap, size_t count) {
  count = std::max<size_t>(count, 1);
  if (*ptr && *cap >= count) return true;
  const size_t want = std::max(count, *cap + *cap / 2);
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  if (cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * want) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  *cap = want;
  return true;
}

// Validate batch items (the checks of sk_batch_create and sk_batch_rebind).
sk_status validate_items(const sk_batch_item* items, int32_t count) {
  if (!items || count < 1) return set_error(SK_ERR_INVALID_ARG, "need at least one item");
  for (int32_t i = 0; i < count; ++i) {
    const sk_batch_item& it = items[i];
    if (!it.A_dev || !it.Y_dev) return set_error(SK_ERR_INVALID_ARG, "item %d: NULL pointer", i);
    if (it.m < 1 || it.n < 1 || it.n > 65535 || it.lda < it.n || it.d < 1 || it.k < 1 || it.k > 64 ||
        it.d % it.k != 0)
      return set_error(SK_ERR_INVALID_ARG, "item %d: invalid sizes (m=%lld n=%lld lda=%lld d=%lld k=%d)", i,
                       (long long)it.m, (long long)it.n, (long long)it.lda, (long long)it.d, it.k);
    if ((reinterpret_cast<uintptr_t>(it.Y_dev) & 3u) != 0)
      return set_error(SK_ERR_INVALID_ARG, "item %d: Y must be 4-byte aligned", i);
    if (it.d / it.k > 0x7fffffffLL) return set_error(SK_ERR_UNSUPPORTED, "item %d: block too large", i);
  }
  return SK_OK;
}

// Build the work list and upload it on `st` (called on the first launch after a create or a rebind,
// so that overrides apply).
sk_status build_batch(sk_batch_s* b, cudaStream_t st) {
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(SK_ERR_CUDA, "cudaGetDevice failed");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  b->device = dev;
  const int32_t threads = b->threads > 0 ? b->threads : 1024;
  const int32_t nwarps = threads / 32;
  // Ring slots hold at most 1 KiB (NC * RB * 4 bytes); two slots per warp are reserved when sizing
  // the accumulators, and the ring gets deeper if the largest accumulator leaves room.
  const size_t optin_c = (size_t)std::min(optin, 232448) - 1024;
  const size_t fixed = (size_t)nwarps * (kWordsPerWarp * 4 + 2 * 1024 + 2 * 8) + 256;
  const size_t budget_floats = (optin_c - fixed) / 4;
  const int32_t count = (int32_t)b->items.size();
  std::vector<BatchDesc> descs(count);
  std::vector<int32_t> ncgs(count), nbgs(count);
  size_t max_floats = 0;
  int32_t slot_max = 128;
  double total_cost = 0.0;
  for (int32_t i = 0; i < count; ++i) {
    const sk_batch_item& it = b->items[i];
    const int64_t B = it.d / it.k;
    const int32_t RB = 32 / ((it.k + 1) / 2);
    // Widest column group (not wider than needed, slot at most 1 KiB) whose accumulator holds all
    // k blocks; if none does, the narrowest width with as many blocks per group as fit.
    int32_t NC = 0, kb = 0;
    const int32_t widths[4] = {32, 16, 8, 4};
    for (int32_t c : widths) {
      if (b->tile_cols > 0 && c != b->tile_cols) continue;
      if (c > 4 && (c / 2 >= it.n || c * RB > 256)) continue;
      if ((size_t)tile_acc_floats((uint32_t)B, it.k, tile_slots(c, it.k), c) <= budget_floats) {
        NC = c;
        kb = it.k;
        break;
      }
    }
    if (NC == 0) {
      NC = b->tile_cols > 0 ? b->tile_cols : 4;
      for (int32_t kbt = it.k; kbt >= 1; --kbt) {
        if ((size_t)tile_acc_floats((uint32_t)B, kbt, tile_slots(NC, kbt), NC) <= budget_floats) {
          kb = kbt;
          break;
        }
      }
    }
    if (kb == 0)
      return set_error(SK_ERR_UNSUPPORTED, "batch item %d: a block of %lld rows does not fit in shared memory", i,
                       (long long)B);
    // One block group: the lane-row path with boxes of several hash rounds (up to 1 KiB), if A's
    // layout allows TMA (decided below, when the maps are encoded).
    const int32_t mb = (kb == it.k) ? std::max(1, std::min(8, 1024 / (RB * NC * 4))) : 1;
    slot_max = std::max(slot_max, ring_slot_bytes(RB * mb, NC));
    BatchDesc& D = descs[i];
    D.D.A = it.A_dev;
    D.D.a_type = kAF32;
    D.D.ldy = 0;
    D.D.Y = it.Y_dev;
    D.D.lda = it.lda;
    D.D.n = it.n;
    D.D.row_base = 0;
    D.D.seed = it.seed;
    D.D.scale = (float)(1.0 / std::sqrt((double)it.k));
    D.D.B = (uint32_t)B;
    D.D.k = (uint32_t)it.k;
    D.D.kp = (uint32_t)((it.k + 1) / 2);
    int l2 = 0;
    while ((1 << l2) < NC) ++l2;
    D.D.log2NC = l2;
    D.D.S = tile_slots(NC, kb);
    D.D.kb = kb;
    D.D.col_off = 0;
    D.D.tmap = nullptr;  // set after the maps are uploaded
    D.D.mb = mb;
    D.D.lr = (kb == it.k) ? 1 : 0;
    D.D.vec = 0;
    ncgs[i] = (int32_t)((it.n + NC - 1) / NC);
    nbgs[i] = (it.k + kb - 1) / kb;
    max_floats = std::max(max_floats, (size_t)tile_acc_floats((uint32_t)B, kb, D.D.S, NC));
    total_cost += (double)it.m * (double)ncgs[i] * NC * it.k;
  }
  // Chunk rows: aim at ~4 work items per CTA slot over the whole batch, and at most 32 chunks per
  // matrix (each output then receives at most 32 rounded contributions).
  const double target_cost = total_cost / (4.0 * sms);
  std::vector<BatchWork> work;
  b->bytes_A = 0;
  for (int32_t i = 0; i < count; ++i) {
    const sk_batch_item& it = b->items[i];
    const int32_t NC = 1 << descs[i].D.log2NC;
    int64_t R;
    if (b->chunk_rows > 0) {
      R = b->chunk_rows;
    } else if (b->item_chunks > 0) {
      R = std::max<int64_t>(4096, (it.m + b->item_chunks - 1) / b->item_chunks);
      R = ((R + 255) / 256) * 256;
    } else {
      const double per_row = (double)ncgs[i] * NC * it.k;
      R = (int64_t)std::ceil(target_cost / std::max(per_row, 1.0));
      R = std::max<int64_t>(R, (it.m + 31) / 32);
      R = std::max<int64_t>(R, 256);
      R = ((R + 255) / 256) * 256;
    }
    descs[i].R = R;
    b->bytes_A += it.m * it.n * 4;
    const int64_t nch = (it.m + R - 1) / R;
    for (int64_t t = 0; t < nch; ++t)
      for (int32_t bg = 0; bg < nbgs[i]; ++bg)
        for (int32_t g = 0; g < ncgs[i]; ++g) {
          BatchWork w;
          w.r0 = t * R;
          w.r1 = std::min((t + 1) * R, it.m);
          w.t = t;
          w.item = i;
          w.g = g;
          w.j0 = bg * descs[i].D.kb;
          w.kbe = std::min(descs[i].D.kb, it.k - w.j0);
          work.push_back(w);
        }
  }
  // Largest first.
  std::stable_sort(work.begin(), work.end(), [&](const BatchWork& x, const BatchWork& y) {
    const double cx = (double)(x.r1 - x.r0) * x.kbe * (1 << descs[x.item].D.log2NC);
    const double cy = (double)(y.r1 - y.r0) * y.kbe * (1 << descs[y.item].D.log2NC);
    return cx > cy;
  });
  std::vector<ZeroSpan>& zs = b->h_zero;
  zs.assign(count, ZeroSpan());
  for (int32_t i = 0; i < count; ++i) {
    const int64_t es = (b->rule == SK_FP32) ? 4 : 2;
    zs[i].p = b->items[i].Y_dev;
    zs[i].bytes = b->items[i].d * b->items[i].n * es;
  }
  // One tensor map per item (A staged through TMA where its layout allows it).
  std::vector<CUtensorMap>& maps = b->h_maps;
  maps.assign(count, CUtensorMap());
  std::vector<int> has_map(count, 0);
  for (int32_t i = 0; i < count; ++i) {
    memset(&maps[i], 0, sizeof(CUtensorMap));
    const sk_batch_item& it = b->items[i];
    has_map[i] = encode_a_map(&maps[i], it.A_dev, kAF32, it.lda, it.n, it.m, 1 << descs[i].D.log2NC,
                              (32 / ((it.k + 1) / 2)) * descs[i].D.mb)
                     ? 1
                     : 0;
    if (!has_map[i]) {
      // direct loads: the target-word path, one hash round per batch
      descs[i].D.mb = 1;
      descs[i].D.lr = 0;
    }
  }
  if (!b->d_status) {
    if (cudaMalloc(&b->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->d_counter, sizeof(int32_t)) != cudaSuccess) {
      free_batch_dev(b);
      cudaGetLastError();
      return set_error(SK_ERR_OOM, "batch status allocation failed");
    }
  }
  if (cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), st) != cudaSuccess)
    return set_error(SK_ERR_CUDA, "batch status reset: %s", cudaGetErrorString(cudaGetLastError()));
  if (!ensure_dev(&b->d_maps, &b->cap_maps, (size_t)count) || !ensure_dev(&b->d_descs, &b->cap_descs, (size_t)count) ||
      !ensure_dev(&b->d_work, &b->cap_work, work.size()) || !ensure_dev(&b->d_zero, &b->cap_zero, (size_t)count)) {
    free_batch_dev(b);
    return set_error(SK_ERR_OOM, "batch work list allocation failed");
  }
  for (int32_t i = 0; i < count; ++i) descs[i].D.tmap = has_map[i] ? (const void*)(b->d_maps + i) : nullptr;
  b->h_descs.swap(descs);
  b->h_work.swap(work);
  cudaError_t eu = cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice, st);
  if (eu == cudaSuccess)
    eu = cudaMemcpyAsync(b->d_descs, b->h_descs.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st);
  if (eu == cudaSuccess && !b->h_work.empty())
    eu = cudaMemcpyAsync(b->d_work, b->h_work.data(), sizeof(BatchWork) * b->h_work.size(), cudaMemcpyHostToDevice, st);
  if (eu == cudaSuccess) eu = cudaMemcpyAsync(b->d_zero, zs.data(), sizeof(ZeroSpan) * count, cudaMemcpyHostToDevice, st);
  if (eu != cudaSuccess) return set_error(SK_ERR_CUDA, "batch work-list upload: %s", cudaGetErrorString(eu));
  b->nwork = (int64_t)b->h_work.size();
  b->acc_floats = (int64_t)max_floats;
  b->slot_bytes = slot_max;
  {
    const size_t base = smem_plan(b->acc_floats, nwarps, slot_max, 0).total;
    const size_t per_depth = (size_t)nwarps * (slot_max + 8);
    int32_t depth = (int32_t)std::min<size_t>(kMaxRingDepth, (optin_c - base) / per_depth);
    b->depth = std::max(1, depth);
  }
  b->smem = smem_plan(b->acc_floats, nwarps, slot_max, b->depth).total;
  b->use_threads = threads;
  const void* kern = batch_kernel_ptr(b->rule);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess)
    return set_error(SK_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(cudaGetLastError()));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, (void (*)(const BatchDesc*, const BatchWork*, int64_t, int32_t*, int64_t, int32_t, int32_t, unsigned*))kern,
      threads, b->smem);
  if (per_sm < 1) return set_error(SK_ERR_UNSUPPORTED, "batch kernel does not fit on an SM");
  b->grid = (int32_t)std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(b->nwork, 1));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SK_ERR_CUDA, "batch build: %s", cudaGetErrorString(e));
  b->built = true;
  return SK_OK;
}

}  // namespace

extern "C" {

sk_status sk_batch_create(const sk_batch_item* items, int32_t count, int32_t rule, sk_batch* out) {
  clear_error();
  if (!out) return set_error(SK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (rule < SK_FP32 || rule > SK_BF16_RN) return set_error(SK_ERR_INVALID_ARG, "unknown rule %d", rule);
  sk_status s = validate_items(items, count);
  if (s != SK_OK) return s;
  sk_batch_s* b = new (std::nothrow) sk_batch_s();
  if (!b) return set_error(SK_ERR_OOM, "host allocation failed");
  b->items.assign(items, items + count);
  b->rule = rule;
  *out = b;
  return SK_OK;
}

sk_status sk_batch_rebind(sk_batch b, const sk_batch_item* items, int32_t count) {
  clear_error();
  if (!b) return set_error(SK_ERR_INVALID_ARG, "batch is NULL");
  sk_status s = validate_items(items, count);
  if (s != SK_OK) return s;
  b->items.assign(items, items + count);
  b->built = false;
  return SK_OK;
}

sk_status sk_batch_set(sk_batch b, int32_t key, int64_t value) {
  clear_error();
  if (!b) return set_error(SK_ERR_INVALID_ARG, "batch is NULL");
  if (b->built) return set_error(SK_ERR_INVALID_ARG, "batch already launched; set parameters before the first launch");
  switch (key) {
    case SK_PARAM_TILE_COLS:
      if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32)
        return set_error(SK_ERR_INVALID_ARG, "tile cols must be 0, 4, 8, 16 or 32");
      b->tile_cols = (int32_t)value;
      return SK_OK;
    case SK_PARAM_THREADS:
      if (value != 0 && (value < 128 || value > 1024 || value % 32 != 0))
        return set_error(SK_ERR_INVALID_ARG, "threads must be 0 or a multiple of 32 in [128, 1024]");
      b->threads = (int32_t)value;
      return SK_OK;
    case SK_PARAM_CHUNK_ROWS:
      if (value < 0) return set_error(SK_ERR_INVALID_ARG, "chunk rows must be >= 0");
      b->chunk_rows = value;
      return SK_OK;
    case SK_PARAM_ITEM_CHUNKS:
      if (value < 0) return set_error(SK_ERR_INVALID_ARG, "chunks per item must be >= 0");
      b->item_chunks = value;
      return SK_OK;
    default:
      return set_error(SK_ERR_INVALID_ARG, "unknown batch key %d", key);
  }
}

sk_status sk_batch_launch(sk_batch b, void* stream) {
  clear_error();
  if (!b) return set_error(SK_ERR_INVALID_ARG, "batch is NULL");
  if (!b->built) {
    sk_status s = build_batch(b, (cudaStream_t)stream);
    if (s != SK_OK) return s;
  }
  int32_t launches = 0;
  cudaError_t e = launch_batch(b->d_descs, b->d_work, b->nwork, b->d_counter, b->d_zero, (int32_t)b->items.size(),
                               b->rule, b->use_threads, b->smem, b->grid, b->acc_floats, b->slot_bytes, b->depth,
                               b->d_status, (cudaStream_t)stream, &launches);
  if (e != cudaSuccess) return set_error(SK_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  return SK_OK;
}

sk_status sk_batch_info(sk_batch b, int64_t* work_items, int64_t* bytes_A) {
  clear_error();
  if (!b) return set_error(SK_ERR_INVALID_ARG, "batch is NULL");
  if (!b->built) {
    sk_status s = build_batch(b, 0);
    if (s != SK_OK) return s;
  }
  if (work_items) *work_items = b->nwork;
  if (bytes_A) *bytes_A = b->bytes_A;
  return SK_OK;
}

void sk_batch_destroy(sk_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch_dev(b);
  delete b;
}

}  // extern "C"
