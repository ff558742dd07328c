// C ABI of libsk: plan objects, argument validation, kernel dispatch, the host-buffer pipeline
// and the sketch-and-solve driver. Declarations and contracts: include/sk.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/sk.h"
#include "sk_hostutil.h"
#include "sk_internal.h"
#include "sk_tile.cuh"

namespace sk {

namespace {
thread_local char g_err[512] = {0};
}

sk_status set_error(sk_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = 0; }

const char* last_error_message() { return g_err; }

}  // namespace sk

using namespace sk;

namespace sk {
sk_status noalloc_read_status(unsigned* out);  // sk_noalloc.cu
}

struct sk_plan_s {
  int64_t d = 0, m = 0, B = 0;
  int32_t k = 0, rule = 0;
  uint64_t seed = 0;
  float scale = 1.f;
  // parameters
  int64_t R = 0;
  int32_t mode = SK_MODE_ATOMIC;
  int64_t row_offset = 0;
  int32_t kernel = SK_KERNEL_AUTO;
  int32_t tile_cols = 0;
  int32_t threads = 0;
  int64_t solve_group_rows = 0;  // rows per QR group of sk_solve (0: as many as shared memory holds)
  int32_t list_cap = 0;          // register kernel: list entries per output row and box (0: automatic)
  int64_t scratch_limit = 0;     // bound on the plan's device scratch in bytes (0: none)
  int64_t solve_wait_cycles = 0; // bound on each grid-barrier wait of the QR kernel (0: default)
  int64_t last_launches = 0, last_R = 0;
  int32_t last_kernel = 0;  // kernel of the last sketch: 1 tile, 2 literal, 3 owner, 4 global, 5 deterministic
  bool last_noalloc = false;  // the last sketch was an sk_apply_noalloc call (status in the static array)
  // device scratch
  float* det_P = nullptr;
  size_t det_P_bytes = 0;
  unsigned* dstatus = nullptr;  // sticky device status word of the sketch kernels
  float* tileP = nullptr;       // two-level chunk totals (zero between launches)
  double* lsqr = nullptr;       // sk_solve_precond: u (m), 8 n-vectors, scalars, x0 (n floats)
  size_t lsqr_bytes = 0;
  size_t tileP_bytes = 0;
  void* solve_buf = nullptr;
  size_t solve_bytes = 0;
  size_t solve_status_off = 0, solve_kappa_off = 0;
  // host-pipeline staging
  float* stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  void* ydev = nullptr;
  size_t ydev_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_used[2] = {nullptr, nullptr};
};

namespace {

constexpr int32_t kMaxK = 64;
constexpr int64_t kMaxN = 65535;
constexpr int32_t kMaxSolveN = 1024;

sk_status cuda_fail(cudaError_t e, const char* what) {
  return set_error(SK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DevInfo {
  int sms = 0, optin = 0;
};

sk_status dev_info(DevInfo* di) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&di->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&di->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return SK_OK;
}

size_t elem_size(int32_t rule) { return rule == SK_FP32 ? 4 : 2; }

// Device scratch the plan holds, in bytes.
size_t plan_scratch_bytes(const sk_plan_s* p) {
  return p->det_P_bytes + (p->dstatus ? sizeof(unsigned) : 0) + p->tileP_bytes + p->lsqr_bytes + p->solve_bytes +
         2 * p->stage_bytes + p->ydev_bytes;
}

// Replace one plan buffer (*ptr of *cur bytes) by a new one of `bytes`: checked against the plan's
// scratch limit first, so a refused call leaves the plan's buffers as they were and enqueues nothing;
// SK_ERR_OOM also when cudaMalloc fails.
template <typename T>
sk_status plan_grow(sk_plan_s* p, T** ptr, size_t* cur, size_t bytes, const char* what) {
  if (p->scratch_limit > 0 && plan_scratch_bytes(p) - *cur + bytes > (size_t)p->scratch_limit)
    return set_error(SK_ERR_OOM, "%s (%zu bytes) would take the plan's scratch above its limit of %lld bytes", what,
                     bytes, (long long)p->scratch_limit);
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cur = 0;
  if (cudaMalloc(reinterpret_cast<void**>(ptr), bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SK_ERR_OOM, "%s (%zu bytes)", what, bytes);
  }
  *cur = bytes;
  return SK_OK;
}

// Tile-kernel configuration for a plan and a column count.
struct TileCfg {
  int32_t NC = 0, kb = 0, threads = 0, grid = 0, slices = 1, depth = 1, mb = 1;
  int64_t R = 0;
  bool serial = false;
  bool lr = false;
  bool own = false;
  bool vec = false;
  bool glob = false;
  bool reg = false;
  int32_t reg_nsub = 0, reg_cap = 0;
};

// Default chunk length: at most 8 chunks per matrix (each output then receives at most 8 rounded
// contributions) and at least 4096 rows per chunk; a multiple of 32.
int64_t default_chunk_rows(int64_t m) {
  int64_t R = std::max<int64_t>(4096, (m + 7) / 8);
  return ((R + 31) / 32) * 32;
}

// Whether A (device pointer, row stride lda, es-byte elements) can be staged through TMA: a
// 16-byte-aligned base and a row stride that is a multiple of 16 bytes.
bool tma_layout_ok(const void* A, int64_t lda, int64_t es = 4) {
  return (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (lda * es) % 16 == 0;
}

// Split each chunk into slices: at least about 4 work items per resident CTA, slices at least
// max(4096, 2d) rows long so the partial flushes (d x NC floats each) stay small, and, among the
// slice counts up to 4x that minimum, the one whose work items fill the last round of CTAs best
// (the items of one launch are of equal size, so a last round of 120 items on 152 CTAs idles 21 % of
// the GPU for a whole item).
int32_t choose_slices(const sk_plan_s* p, int64_t rows, int64_t R, int64_t ncg, int64_t nbg, int32_t cps,
                      const DevInfo& di) {
  const int64_t first = ((p->row_offset % R) + R) % R;  // offset of the first row inside its chunk
  const int64_t chunks = (first + rows + R - 1) / R;
  const int64_t G = (int64_t)di.sms * std::max(cps, 1);
  const int64_t per = std::max<int64_t>(1, chunks * ncg * nbg);
  const int64_t s_lo = std::max<int64_t>(1, (4 * G + per - 1) / per);
  const int64_t min_rows = std::max<int64_t>(4096, 2 * p->d);
  const int64_t s_max = std::min<int64_t>(std::max<int64_t>(1, std::min(R, rows) / min_rows), 4096);
  int64_t best = std::min(s_lo, s_max);
  double best_waste = 1e30;
  for (int64_t sl = std::min(s_lo, s_max); sl <= std::min(4 * s_lo, s_max); ++sl) {
    const int64_t items = per * sl;
    const double waste = (double)((items + G - 1) / G * G) / (double)items;
    if (waste < best_waste - 0.005) {
      best_waste = waste;
      best = sl;
    }
  }
  return (int32_t)best;
}

// Owner-kernel configuration (atomic mode, SK_KERNEL_OWNER): blocks per item kb = 2 when two blocks
// of 32-column lines fit in shared memory, else 1; false if the kernel does not apply.
bool choose_own(const sk_plan_s* p, int64_t n, int64_t rows, const DevInfo& di, bool tma_ok, TileCfg* cfg) {
  if (p->mode != SK_MODE_ATOMIC || !tma_ok || n < 32 || rows >= ((int64_t)1 << 31)) return false;
  if (p->kernel != SK_KERNEL_OWNER) return false;
  const size_t optin = (size_t)std::min(di.optin, 232448) - 1024;
  int32_t kb = 0;
  if (p->k >= 2 && own_smem_bytes(p->B, 2) <= optin) kb = 2;
  else if (own_smem_bytes(p->B, 1) <= optin) kb = 1;
  if (kb == 0) return false;
  const int64_t R = p->R > 0 ? p->R : default_chunk_rows(p->m);
  const int32_t cps = own_ctas_per_sm(p->rule, own_smem_bytes(p->B, kb));
  if (cps < 1) return false;
  const int64_t ncg = (n + 31) / 32;
  const int64_t nbg = (p->k + kb - 1) / kb;
  cfg->NC = 32;
  cfg->kb = kb;
  cfg->threads = own_threads();
  cfg->grid = 0;
  cfg->R = R;
  cfg->slices = choose_slices(p, rows, R, ncg, nbg, cps, di);
  cfg->depth = 1;
  cfg->mb = 1;
  cfg->serial = false;
  cfg->lr = false;
  cfg->own = true;
  cfg->vec = false;
  return true;
}

// Global-accumulator configuration: chunk totals in device memory (any block height).
void choose_global(const sk_plan_s* p, TileCfg* cfg) {
  *cfg = TileCfg();
  cfg->NC = 4;
  cfg->kb = p->k;
  cfg->threads = 256;
  cfg->R = p->R > 0 ? p->R : default_chunk_rows(p->m);
  cfg->slices = 1;
  cfg->glob = true;
}

// Register-kernel configuration (atomic mode, FP32 A staged through TMA): the staged box and list
// capacity for the plan's block height, the default chunk length and the slice count. AUTO takes it
// for k >= 2, n >= 32 and blocks of at most 512 rows (not n >= 256 with k = 2, which goes to the
// global kernel), where it is faster than the tile kernel
// (measured at 2^22 x 64: d = 4096, k = 8: 1060 vs 818 GB/s; d = 1024, k = 8: 1520 vs 798; at
// d = 4096 with k = 4 or 2 (B = 1024, 2048) the tile kernel stays ahead: 1416 vs 1357, 1735 vs 1448).
bool choose_reg(const sk_plan_s* p, int64_t n, int64_t rows, const DevInfo& di, bool tma_ok, bool a_fp32,
                TileCfg* cfg) {
  if (p->mode != SK_MODE_ATOMIC || !tma_ok || !a_fp32 || rows >= ((int64_t)1 << 31)) return false;
  if (p->kernel == SK_KERNEL_AUTO) {
    if (p->tile_cols != 0 || p->threads != 0 || p->k < 2 || n < 32 || p->B > 512) return false;
    if (n >= 256 && p->k <= 2) return false;  // the global kernel's case (wide rows, few nonzeros)
  } else if (p->kernel != SK_KERNEL_REGISTER) {
    return false;
  }
  const size_t optin = (size_t)std::min(di.optin, 232448) - 1024;
  int32_t nsub = 0, cap = 0;
  if (!reg_choose_box(p->d, p->B, optin, p->list_cap, &nsub, &cap)) return false;
  const int64_t R = p->R > 0 ? p->R : default_chunk_rows(p->m);
  const int64_t ncg = (n + 31) / 32;
  const int64_t ntg = (p->d + reg_targets() - 1) / reg_targets();
  *cfg = TileCfg();
  cfg->NC = 32;
  cfg->kb = p->k;
  cfg->threads = reg_threads();
  cfg->R = R;
  cfg->slices = choose_slices(p, rows, R, ncg, ntg, 1, di);
  cfg->reg = true;
  cfg->reg_nsub = nsub;
  cfg->reg_cap = cap;
  return true;
}

sk_status choose_tile(const sk_plan_s* p, int64_t n, int64_t rows, const DevInfo& di, TileCfg* cfg,
                      bool tma_ok = false, bool a_fp32 = true) {
  if (choose_reg(p, n, rows, di, tma_ok, a_fp32, cfg)) return SK_OK;
  if (p->kernel == SK_KERNEL_REGISTER)
    return set_error(SK_ERR_UNSUPPORTED,
                     "register kernel: needs atomic mode, FP32 A, A 16-byte aligned with lda %% 4 == 0 and fewer "
                     "than 2^31 rows");
  if (p->kernel == SK_KERNEL_GLOBAL) {
    if (p->mode != SK_MODE_ATOMIC) return set_error(SK_ERR_UNSUPPORTED, "the global kernel runs in atomic mode only");
    choose_global(p, cfg);
    return SK_OK;
  }
  if (choose_own(p, n, rows, di, tma_ok, cfg)) return SK_OK;
  if (p->kernel == SK_KERNEL_OWNER)
    return set_error(SK_ERR_UNSUPPORTED,
                     "owner kernel: needs atomic mode, n >= 32, A 16-byte aligned with lda %% 4 == 0 and "
                     "2 x %lld x 128 bytes of shared memory",
                     (long long)p->B);
  const bool serial = (p->mode == SK_MODE_SERIAL_TILE);
  if (n == 1 && !serial && p->tile_cols <= 4) {
    // A single column: the vector path (one thread per row, accumulator lines of one quad).
    const int32_t threads = p->threads > 0 ? p->threads : 1024;
    int32_t kb = 0;
    for (int32_t kbt = p->k; kbt >= 1; --kbt) {
      const int64_t fl = tile_acc_floats((uint32_t)p->B, kbt, tile_slots(4, kbt), 4);
      if (tile_smem_bytes(p->B, kbt, 4, threads, p->k, 1) <= (size_t)std::min(di.optin, 232448) - 1024 && fl < (1 << 29)) {
        kb = kbt;
        break;
      }
    }
    if (kb > 0) {
      const int64_t R = p->R > 0 ? p->R : default_chunk_rows(p->m);
      const int64_t nbg = (p->k + kb - 1) / kb;
      const int32_t cps = tile_ctas_per_sm(p->rule, threads, tile_smem_bytes(p->B, kb, 4, threads, p->k, 1));
      cfg->NC = 4;
      cfg->kb = kb;
      cfg->threads = threads;
      cfg->grid = 0;
      cfg->R = R;
      cfg->slices = choose_slices(p, rows, R, 1, nbg, cps, di);
      cfg->depth = 1;
      cfg->mb = 1;
      cfg->serial = false;
      cfg->lr = false;
      cfg->own = false;
      cfg->vec = true;
      return SK_OK;
    }
  }
  const int32_t threads = serial ? 32 : (p->threads > 0 ? p->threads : 1024);
  const int32_t nwarps = threads / 32;
  const int32_t RB = 32 / ((p->k + 1) / 2);
  const size_t optin = (size_t)std::min(di.optin, 232448) - 1024;
  // Fits: accumulator + target words + a ring of at least one slot per warp.
  auto fits = [&](int32_t c, int32_t kbt) {
    const int64_t fl = tile_acc_floats((uint32_t)p->B, kbt, tile_slots(c, kbt), c);
    return tile_smem_bytes(p->B, kbt, c, threads, p->k, 1) <= optin && fl < (1 << 29);
  };
  const int32_t widths[4] = {32, 16, 8, 4};
  int32_t NC = 0, kb = 0;
  for (int32_t c : widths) {
    if (p->tile_cols > 0 && c != p->tile_cols) continue;
    if (!serial && c > 4 && (c / 2 >= n || c * RB > 256)) continue;
    // Serial (verification) mode needs the lane groups of a pass to hit distinct blocks.
    if (serial && (32 / c > p->k || p->k % (32 / c) != 0)) continue;
    if (fits(c, p->k)) {
      NC = c;
      kb = p->k;
      break;
    }
  }
  if (NC == 0 && !serial) {
    NC = p->tile_cols > 0 ? p->tile_cols : 4;
    for (int32_t kbt = p->k; kbt >= 1; --kbt) {
      if (fits(NC, kbt)) {
        kb = kbt;
        break;
      }
    }
  }
  if (NC == 0 || kb == 0) {
    // A block too tall for the on-chip accumulator: chunk totals in device memory instead.
    if (!serial && p->kernel == SK_KERNEL_AUTO) {
      choose_global(p, cfg);
      return SK_OK;
    }
    return set_error(SK_ERR_UNSUPPORTED,
                     "tile kernel: a block of %lld rows does not fit in shared memory with the requested width",
                     (long long)p->B);
  }
  // Where the tile kernel would need several block groups (the target-word scatter, 5-7x slower
  // than the global kernel at n = 1024 and d >= 16384), or only 4-column items for a wide matrix
  // (each row's hash evaluated n/4 times), AUTO takes the global-accumulator kernel. So it does for
  // wide matrices at k <= 2: there the tile kernel's cost is the per-item overhead (hash and staging
  // per column group for only k * NC updates per row) while the global kernel's k n / 4 L2
  // reductions per row are few (measured at n = 256 / 1024, d/n = 2: k = 1 1809 -> 3100 and
  // 2035 -> 3745 GB/s, k = 2 1559 -> 2504 and 1810 -> 2686 GB/s; at k = 4 the two are within 3 %).
  if (!serial && p->kernel == SK_KERNEL_AUTO && p->tile_cols == 0 &&
      (kb < p->k || (NC <= 4 && n >= 256) || (p->k <= 2 && n >= 256))) {
    choose_global(p, cfg);
    return SK_OK;
  }
  // One block group (outside serial mode): every work item takes the lane-row path, with several
  // hash rounds per TMA box (boxes of up to 1 KiB).
  const bool lr = !serial && kb == p->k;
  int32_t mb = 1;
  if (lr) mb = std::max(1, std::min(8, 1024 / (RB * NC * 4)));
  while (mb > 1 && tile_smem_bytes(p->B, kb, NC, threads, p->k, 1, mb) > optin) mb /= 2;
  int32_t depth = 1;
  while (depth < kMaxRingDepth && tile_smem_bytes(p->B, kb, NC, threads, p->k, depth + 1, mb) <= optin) ++depth;
  int64_t R = p->R > 0 ? p->R : default_chunk_rows(p->m);
  int32_t slices = 1;
  if (!serial) {
    const int64_t ncg = (n + NC - 1) / NC;
    const int64_t nbg = (p->k + kb - 1) / kb;
    const int32_t cps = tile_ctas_per_sm(p->rule, threads, tile_smem_bytes(p->B, kb, NC, threads, p->k, depth, mb));
    slices = choose_slices(p, rows, R, ncg, nbg, cps, di);
  }
  cfg->NC = NC;
  cfg->kb = kb;
  cfg->threads = threads;
  cfg->grid = serial ? 1 : 0;
  cfg->R = R;
  cfg->slices = slices;
  cfg->depth = depth;
  cfg->mb = mb;
  cfg->lr = lr;
  cfg->own = false;
  cfg->vec = false;
  cfg->serial = serial;
  return SK_OK;
}

sk_status validate_apply(const sk_plan_s* p, const void* A, int64_t lda, int64_t n, const void* Y,
                         uintptr_t a_align = 4) {
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  if (!A) return set_error(SK_ERR_INVALID_ARG, "A is NULL");
  if (!Y) return set_error(SK_ERR_INVALID_ARG, "Y is NULL");
  if (n < 1 || n > kMaxN) return set_error(SK_ERR_INVALID_ARG, "n=%lld outside [1, %lld]", (long long)n, (long long)kMaxN);
  if (lda < n) return set_error(SK_ERR_INVALID_ARG, "lda=%lld < n=%lld", (long long)lda, (long long)n);
  if ((reinterpret_cast<uintptr_t>(A) & (a_align - 1)) != 0)
    return set_error(SK_ERR_INVALID_ARG, "A must be %d-byte aligned", (int)a_align);
  if ((reinterpret_cast<uintptr_t>(Y) & 3u) != 0) return set_error(SK_ERR_INVALID_ARG, "Y must be 4-byte aligned");
  if (p->m > (int64_t)1 << 40 || lda > ((int64_t)1 << 40) / std::max<int64_t>(p->m, 1))
    return set_error(SK_ERR_UNSUPPORTED, "A larger than 2^40 elements");
  return SK_OK;
}

// Enqueue Y = S * A for rows [row_begin, row_begin + rows) (A row 0 = row_begin) with chunk rows R.
// Y must already be zero, or zero_y set: then Y is zeroed on the stream once the plan's scratch is in
// place (a call refused for lack of scratch leaves Y untouched). a_type: element type of A
// (SK_A_FP32, SK_A_FP16, SK_A_BF16).
sk_status enqueue_sketch(sk_plan_s* p, const void* A, int64_t lda, int64_t n, int64_t row_begin, int64_t rows, void* Y,
                         int64_t R_fixed, cudaStream_t st, int32_t* launches, int64_t* R_used, int64_t col_off = 0,
                         int32_t a_type = SK_A_FP32, bool zero_y = false) {
  p->last_noalloc = false;
  DevInfo di;
  sk_status s = dev_info(&di);
  if (s != SK_OK) return s;
  const int64_t row_end = row_begin + rows;
  const bool literal = (p->kernel == SK_KERNEL_LITERAL);
  if (p->mode == SK_MODE_DETERMINISTIC) {
    int64_t R = R_fixed > 0 ? R_fixed : p->R;
    if (R <= 0) {
      TileCfg cfg;
      s = choose_tile(p, n, p->m, di, &cfg);
      if (s != SK_OK) return s;
      R = literal ? 1 : cfg.R;
    }
    const size_t need = sizeof(float) * (size_t)(p->d * n);
    if (p->det_P_bytes < need) {
      s = plan_grow(p, &p->det_P, &p->det_P_bytes, need, "deterministic-mode scratch");
      if (s != SK_OK) return s;
    }
    if (zero_y) {
      cudaError_t ez = cudaMemsetAsync(Y, 0, elem_size(p->rule) * (size_t)(p->d * n), st);
      if (ez != cudaSuccess) return cuda_fail(ez, "zeroing Y");
    }
    DetLaunch L;
    L.A = A;
    L.a_type = a_type;
    L.Y = Y;
    L.P = p->det_P;
    L.lda = lda;
    L.n = n;
    L.row_begin = row_begin;
    L.row_end = row_end;
    L.d = p->d;
    L.k = p->k;
    L.rule = p->rule;
    L.seed = p->seed;
    L.scale = p->scale;
    L.R = R;
    L.col_off = col_off;
    cudaError_t e = launch_det(L, st, launches);
    if (e != cudaSuccess) return cuda_fail(e, "deterministic kernel launch");
    p->last_kernel = 5;
    if (R_used) *R_used = R;
    return SK_OK;
  }
  if (literal) {
    if (p->R > 1 || R_fixed > 1) return set_error(SK_ERR_INVALID_ARG, "the literal kernel implements chunk rows R = 1 only");
    if (zero_y) {
      cudaError_t ez = cudaMemsetAsync(Y, 0, elem_size(p->rule) * (size_t)(p->d * n), st);
      if (ez != cudaSuccess) return cuda_fail(ez, "zeroing Y");
    }
    LiteralLaunch L;
    L.A = A;
    L.a_type = a_type;
    L.Y = Y;
    L.lda = lda;
    L.n = n;
    L.row_begin = row_begin;
    L.row_end = row_end;
    L.d = p->d;
    L.k = p->k;
    L.rule = p->rule;
    L.seed = p->seed;
    L.scale = p->scale;
    L.col_off = col_off;
    cudaError_t e = launch_literal(L, st, launches);
    if (e != cudaSuccess) return cuda_fail(e, "literal kernel launch");
    p->last_kernel = SK_KERNEL_LITERAL;
    if (R_used) *R_used = 1;
    return SK_OK;
  }
  TileCfg cfg;
  s = choose_tile(p, n, rows, di, &cfg, tma_layout_ok(A, lda, a_type == SK_A_FP32 ? 4 : 2), a_type == SK_A_FP32);
  if (s != SK_OK) return s;
  if (cfg.own && a_type != SK_A_FP32) return set_error(SK_ERR_UNSUPPORTED, "the owner kernel reads FP32 A only");
  if (R_fixed > 0) cfg.R = R_fixed;
  TileLaunch L;
  L.A = A;
  L.a_type = a_type;
  L.Y = Y;
  L.lda = lda;
  L.n = n;
  L.row_begin = row_begin;
  L.row_end = row_end;
  L.d = p->d;
  L.k = p->k;
  L.rule = p->rule;
  L.seed = p->seed;
  L.scale = p->scale;
  L.R = cfg.R;
  L.NC = cfg.NC;
  L.kb = cfg.kb;
  L.threads = cfg.threads;
  L.grid = cfg.grid;
  L.slices = cfg.slices;
  L.depth = cfg.depth;
  L.mb = cfg.mb;
  L.lr = cfg.lr ? 1 : 0;
  L.own = cfg.own ? 1 : 0;
  L.vec = cfg.vec ? 1 : 0;
  L.glob = cfg.glob ? 1 : 0;
  L.reg = cfg.reg ? 1 : 0;
  L.reg_nsub = cfg.reg_nsub;
  L.reg_cap = cfg.reg_cap;
  L.col_off = col_off;
  L.allow_tma = cfg.vec ? 0 : 1;
  if (!p->dstatus) {
    size_t cur = 0;
    s = plan_grow(p, &p->dstatus, &cur, sizeof(unsigned), "status word");
    if (s != SK_OK) return s;
    cudaError_t ez = cudaMemsetAsync(p->dstatus, 0, sizeof(unsigned), st);
    if (ez != cudaSuccess) return cuda_fail(ez, "zeroing status word");
  }
  L.status = p->dstatus;
  L.P = nullptr;
  if (cfg.slices > 1 || cfg.glob || cfg.reg) {
    const size_t needP = sizeof(float) * (size_t)launch_P_floats(L);
    if (p->tileP_bytes < needP) {
      s = plan_grow(p, &p->tileP, &p->tileP_bytes, needP, "chunk-total scratch");
      if (s != SK_OK) return s;
      cudaError_t ez = cudaMemsetAsync(p->tileP, 0, needP, st);
      if (ez != cudaSuccess) return cuda_fail(ez, "zeroing chunk totals");
    }
    L.P = p->tileP;
  }
  if (zero_y) {
    cudaError_t ez = cudaMemsetAsync(Y, 0, elem_size(p->rule) * (size_t)(p->d * n), st);
    if (ez != cudaSuccess) return cuda_fail(ez, "zeroing Y");
  }
  cudaError_t e = launch_tile(L, st, launches);
  if (e != cudaSuccess)
    return cuda_fail(e, cfg.glob  ? "global kernel launch"
                        : cfg.reg ? "register kernel launch"
                        : cfg.own ? "owner kernel launch"
                                  : "tile kernel launch");
  p->last_kernel = cfg.glob ? SK_KERNEL_GLOBAL : cfg.reg ? SK_KERNEL_REGISTER : cfg.own ? SK_KERNEL_OWNER : SK_KERNEL_TILE;
  if (R_used) *R_used = cfg.R;
  return SK_OK;
}

}  // namespace

extern "C" {

int32_t sk_version(void) { return 10000; }

const char* sk_last_error(void) { return last_error_message(); }

sk_status sk_plan_create(int64_t d, int64_t m, int32_t k, int32_t rule, uint64_t seed, sk_plan* out) {
  clear_error();
  if (!out) return set_error(SK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > kMaxK) return set_error(SK_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, kMaxK);
  if (d < 1 || d % k != 0) return set_error(SK_ERR_INVALID_ARG, "d=%lld must be a positive multiple of k=%d", (long long)d, k);
  if (d > 0x7fffffffLL) return set_error(SK_ERR_UNSUPPORTED, "d=%lld above 2^31-1", (long long)d);
  if (m < 1) return set_error(SK_ERR_INVALID_ARG, "m=%lld must be >= 1", (long long)m);
  if (m > ((int64_t)1 << 56)) return set_error(SK_ERR_UNSUPPORTED, "m=%lld too large", (long long)m);
  if (rule < SK_FP32 || rule > SK_BF16_RN) return set_error(SK_ERR_INVALID_ARG, "unknown rule %d", rule);
  sk_plan_s* p = new (std::nothrow) sk_plan_s();
  if (!p) return set_error(SK_ERR_OOM, "host allocation failed");
  p->d = d;
  p->m = m;
  p->k = k;
  p->B = d / k;
  p->rule = rule;
  p->seed = seed;
  p->scale = (float)(1.0 / std::sqrt((double)k));
  *out = p;
  return SK_OK;
}

sk_status sk_plan_set(sk_plan p, int32_t key, int64_t v) {
  clear_error();
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  switch (key) {
    case SK_PARAM_CHUNK_ROWS:
      if (v < 0) return set_error(SK_ERR_INVALID_ARG, "chunk rows must be >= 0");
      p->R = v;
      return SK_OK;
    case SK_PARAM_MODE:
      if (v < 0 || v > 2) return set_error(SK_ERR_INVALID_ARG, "mode must be 0 (atomic), 1 (deterministic) or 2 (serial tile)");
      p->mode = (int32_t)v;
      return SK_OK;
    case SK_PARAM_ROW_OFFSET:
      if (v < 0) return set_error(SK_ERR_INVALID_ARG, "row offset must be >= 0");
      p->row_offset = v;
      return SK_OK;
    case SK_PARAM_KERNEL:
      if (v < SK_KERNEL_AUTO || (v > SK_KERNEL_GLOBAL && v != SK_KERNEL_REGISTER))
        return set_error(SK_ERR_INVALID_ARG, "unknown kernel %lld", (long long)v);
      p->kernel = (int32_t)v;
      return SK_OK;
    case SK_PARAM_TILE_COLS:
      if (v != 0 && v != 4 && v != 8 && v != 16 && v != 32)
        return set_error(SK_ERR_INVALID_ARG, "tile cols must be 0, 4, 8, 16 or 32");
      p->tile_cols = (int32_t)v;
      return SK_OK;
    case SK_PARAM_THREADS:
      if (v != 0 && (v < 128 || v > 1024 || v % 32 != 0))
        return set_error(SK_ERR_INVALID_ARG, "threads must be 0 or a multiple of 32 in [128, 1024]");
      p->threads = (int32_t)v;
      return SK_OK;
    case SK_PARAM_SOLVE_GROUP_ROWS:
      if (v < 0) return set_error(SK_ERR_INVALID_ARG, "solve group rows must be >= 0");
      p->solve_group_rows = v;
      return SK_OK;
    case SK_PARAM_LIST_CAP:
      if (v < 0 || v > 64) return set_error(SK_ERR_INVALID_ARG, "list capacity must be in [0, 64]");
      p->list_cap = (int32_t)v;
      return SK_OK;
    case SK_PARAM_ROWS:
      if (v < 1) return set_error(SK_ERR_INVALID_ARG, "rows must be >= 1");
      if (v > ((int64_t)1 << 56)) return set_error(SK_ERR_UNSUPPORTED, "rows=%lld too large", (long long)v);
      p->m = v;
      return SK_OK;
    case SK_PARAM_SCRATCH_LIMIT:
      if (v < 0) return set_error(SK_ERR_INVALID_ARG, "scratch limit must be >= 0");
      p->scratch_limit = v;
      return SK_OK;
    case SK_PARAM_SOLVE_WAIT_CYCLES:
      if (v < 0) return set_error(SK_ERR_INVALID_ARG, "solve wait cycles must be >= 0");
      p->solve_wait_cycles = v;
      return SK_OK;
    default:
      return set_error(SK_ERR_INVALID_ARG, "unknown or read-only key %d", key);
  }
}

sk_status sk_plan_get(sk_plan p, int32_t key, int64_t* v) {
  clear_error();
  if (!p || !v) return set_error(SK_ERR_INVALID_ARG, "NULL argument");
  switch (key) {
    case SK_PARAM_CHUNK_ROWS: *v = p->R; return SK_OK;
    case SK_PARAM_MODE: *v = p->mode; return SK_OK;
    case SK_PARAM_ROW_OFFSET: *v = p->row_offset; return SK_OK;
    case SK_PARAM_KERNEL: *v = p->kernel; return SK_OK;
    case SK_PARAM_TILE_COLS: *v = p->tile_cols; return SK_OK;
    case SK_PARAM_THREADS: *v = p->threads; return SK_OK;
    case SK_PARAM_SOLVE_GROUP_ROWS: *v = p->solve_group_rows; return SK_OK;
    case SK_PARAM_LIST_CAP: *v = p->list_cap; return SK_OK;
    case SK_PARAM_SCRATCH_LIMIT: *v = p->scratch_limit; return SK_OK;
    case SK_PARAM_ROWS: *v = p->m; return SK_OK;
    case SK_PARAM_SOLVE_WAIT_CYCLES: *v = p->solve_wait_cycles; return SK_OK;
    case SK_PARAM_SCRATCH_BYTES: *v = (int64_t)plan_scratch_bytes(p); return SK_OK;
    case SK_PARAM_LAST_LAUNCHES: *v = p->last_launches; return SK_OK;
    case SK_PARAM_LAST_CHUNK_ROWS: *v = p->last_R; return SK_OK;
    case SK_PARAM_LAST_KERNEL: *v = p->last_kernel; return SK_OK;
    case SK_PARAM_DEVICE_STATUS: {
      *v = 0;
      if (!p->dstatus && !p->last_noalloc) return SK_OK;
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "device status");
      unsigned w = 0;
      if (p->dstatus) {
        e = cudaMemcpy(&w, p->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "device status");
      }
      if (p->last_noalloc) {
        unsigned wn = 0;
        sk_status s = noalloc_read_status(&wn);
        if (s != SK_OK) return s;
        w |= wn;
      }
      *v = (int64_t)w;
      return SK_OK;
    }
    default: return set_error(SK_ERR_INVALID_ARG, "unknown key %d", key);
  }
}

sk_status sk_apply(sk_plan p, const float* A, int64_t lda, int64_t n, void* Y, void* stream) {
  clear_error();
  sk_status s = validate_apply(p, A, lda, n, Y);
  if (s != SK_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t launches = 0;
  int64_t R_used = 0;
  s = enqueue_sketch(p, A, lda, n, p->row_offset, p->m, Y, 0, st, &launches, &R_used, 0, SK_A_FP32, true);
  p->last_launches = launches;
  p->last_R = R_used;
  return s;
}

sk_status sk_apply_typed(sk_plan p, const void* A, int32_t a_type, int64_t lda, int64_t n, void* Y, void* stream) {
  clear_error();
  if (a_type != SK_A_FP32 && a_type != SK_A_FP16 && a_type != SK_A_BF16)
    return set_error(SK_ERR_INVALID_ARG, "unknown element type %d of A", a_type);
  sk_status s = validate_apply(p, A, lda, n, Y, a_type == SK_A_FP32 ? 4 : 2);
  if (s != SK_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t launches = 0;
  int64_t R_used = 0;
  s = enqueue_sketch(p, A, lda, n, p->row_offset, p->m, Y, 0, st, &launches, &R_used, 0, a_type, true);
  p->last_launches = launches;
  p->last_R = R_used;
  return s;
}

sk_status sk_apply_host(sk_plan p, const float* A_host, int64_t lda, int64_t n, void* Y_host, void* stream) {
  clear_error();
  sk_status s = validate_apply(p, A_host, lda, n, Y_host);
  if (s != SK_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  DevInfo di;
  s = dev_info(&di);
  if (s != SK_OK) return s;
  // Chunk rows of the whole matrix, so that the tiles reproduce sk_apply's chunks exactly.
  int64_t R = p->R;
  if (p->kernel == SK_KERNEL_LITERAL) R = 1;
  if (R <= 0) {
    TileCfg cfg;
    s = choose_tile(p, n, p->m, di, &cfg);
    if (s != SK_OK) return s;
    R = cfg.R;
  }
  // Tiles of whole chunks, about 128 MiB each.
  const int64_t row_bytes = lda * 4;
  const int64_t target_rows = std::max<int64_t>(1, ((int64_t)128 << 20) / row_bytes);
  int64_t tile_rows;
  if (R >= target_rows) {
    tile_rows = R;
  } else {
    tile_rows = (target_rows / R) * R;
  }
  // The first chunk may be partial when the row offset is not a multiple of R: align tiles to the
  // global chunk grid.
  tile_rows = std::min(tile_rows, p->m + (p->row_offset % R));
  const size_t tile_bytes = (size_t)tile_rows * (size_t)row_bytes;
  const size_t ybytes = elem_size(p->rule) * (size_t)(p->d * n);
  if (p->stage_bytes < tile_bytes) {
    // both staging tiles at once against the limit (plan_grow counts stage_bytes twice)
    if (p->scratch_limit > 0 && plan_scratch_bytes(p) - 2 * p->stage_bytes + 2 * tile_bytes > (size_t)p->scratch_limit)
      return set_error(SK_ERR_OOM, "host pipeline staging (2 x %zu bytes) would take the plan's scratch above its limit",
                       tile_bytes);
    for (int b = 0; b < 2; ++b) {
      if (p->stage[b]) cudaFree(p->stage[b]);
      p->stage[b] = nullptr;
    }
    p->stage_bytes = 0;
    for (int b = 0; b < 2; ++b) {
      if (cudaMalloc(&p->stage[b], tile_bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(SK_ERR_OOM, "host pipeline staging (%zu bytes)", tile_bytes);
      }
    }
    p->stage_bytes = tile_bytes;
  }
  if (p->ydev_bytes < ybytes) {
    s = plan_grow(p, &p->ydev, &p->ydev_bytes, ybytes, "host pipeline Y buffer");
    if (s != SK_OK) return s;
  }
  if (!p->copy_stream) {
    if (cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "copy stream");
    for (int b = 0; b < 2; ++b) {
      cudaEventCreateWithFlags(&p->ev_copied[b], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&p->ev_used[b], cudaEventDisableTiming);
    }
  }
  int32_t launches = 0;
  cudaError_t e = cudaMemsetAsync(p->ydev, 0, ybytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing Y");
  // Buffers start free: mark both as used-and-finished on the compute stream.
  for (int b = 0; b < 2; ++b) cudaEventRecord(p->ev_used[b], st);
  int64_t done = 0;
  int which = 0;
  const int64_t g0 = p->row_offset;
  while (done < p->m) {
    // Tile boundaries on the global chunk grid.
    const int64_t gstart = g0 + done;
    const int64_t chunk_start = (gstart / R) * R;
    int64_t gend = chunk_start + tile_rows;
    if (gend <= gstart) gend = gstart + R;
    gend = std::min(gend, g0 + p->m);
    const int64_t rows = gend - gstart;
    float* buf = p->stage[which];
    e = cudaStreamWaitEvent(p->copy_stream, p->ev_used[which], 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline wait");
    if (lda == n) {
      e = cudaMemcpyAsync(buf, A_host + done * lda, (size_t)rows * n * 4, cudaMemcpyHostToDevice, p->copy_stream);
    } else {
      e = cudaMemcpy2DAsync(buf, (size_t)lda * 4, A_host + done * lda, (size_t)lda * 4, (size_t)n * 4, (size_t)rows,
                            cudaMemcpyHostToDevice, p->copy_stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host to device copy");
    cudaEventRecord(p->ev_copied[which], p->copy_stream);
    cudaStreamWaitEvent(st, p->ev_copied[which], 0);
    s = enqueue_sketch(p, buf, lda, n, gstart, rows, p->ydev, R, st, &launches, nullptr);
    if (s != SK_OK) return s;
    cudaEventRecord(p->ev_used[which], st);
    done += rows;
    which ^= 1;
  }
  e = cudaMemcpyAsync(Y_host, p->ydev, ybytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sk_apply_host");
  p->last_launches = launches;
  p->last_R = R;
  return SK_OK;
}

sk_status sk_materialize_S(sk_plan p, int64_t i0, int64_t cnt, int32_t* rows, int8_t* signs, void* stream) {
  clear_error();
  if (!p || !rows || !signs) return set_error(SK_ERR_INVALID_ARG, "NULL argument");
  if (i0 < 0 || cnt < 0) return set_error(SK_ERR_INVALID_ARG, "negative range");
  if (cnt == 0) return SK_OK;
  cudaError_t e = launch_pattern(p->d, p->k, p->seed, i0, cnt, rows, signs, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pattern kernel launch");
  return SK_OK;
}

// Solve scratch layout (bytes, each region 256-byte aligned):
//   Y_A (d*n elements), Y_b (d elements), part (n + n*(n+1) doubles), R (n*(n+1) doubles),
//   bcast (n doubles), bar (grid-barrier counters), status (1 word), kappa (1 double).
namespace {
struct SolveLayout {
  size_t ya, yb, part, R, bcast, bar, status, kappa, stack[2], total;
};
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
// stack_groups: groups of the first tree level (0: the sketch is factored by one launch).
SolveLayout solve_layout(int64_t d, int64_t n, int32_t rule, int64_t stack_groups) {
  SolveLayout L;
  size_t off = 0;
  const size_t es = elem_size(rule);
  L.ya = off; off = al256(off + es * (size_t)(d * n));
  L.yb = off; off = al256(off + es * (size_t)d);
  L.part = off; off = al256(off + 8 * (size_t)(n + n * (n + 1)));
  L.R = off; off = al256(off + 8 * (size_t)(n * (n + 1)));
  L.bcast = off; off = al256(off + 8 * (size_t)n);
  L.bar = off; off = al256(off + solve_bar_bytes());
  L.status = off; off = al256(off + 4);
  L.kappa = off; off = al256(off + 8);
  for (int i = 0; i < 2; ++i) {
    L.stack[i] = off;
    off = al256(off + 8 * (size_t)(stack_groups * n * (n + 1)));
  }
  L.total = off;
  return L;
}

// Rows per group of the QR tree for a d x (n+1) sketch: the whole sketch if it fits one launch,
// else a cap of at least 2n rows (each level then shrinks the stack at least by half). 0: unsupported.
int64_t solve_group_cap(const sk_plan_s* p, int64_t n, const DevInfo& di) {
  const int64_t cap_auto = solve_rows_cap(n, di.sms, (size_t)di.optin);
  if (cap_auto < n) return 0;
  int64_t cap = cap_auto;
  if (p->solve_group_rows > 0) cap = std::min(cap, std::max(p->solve_group_rows, 2 * n));
  if (p->d > cap && cap < 2 * n) return 0;
  return cap;
}

// QR back end of sketch-and-solve (paper Sec. 5.3: QR of the sketch SA, then R x = (Q^T Sb)[:n]):
// x from the sketch columns SA (d x n, row stride lda_sa) and Sb (d values, stride sb_stride) in the
// plan's element type, in FP64; tree levels (groups of at most `cap` rows factored, their [R | c]
// factors stacked and factored again) when the sketch is taller than one QR launch holds.
sk_status solve_backend(sk_plan_s* p, const void* SA, int64_t lda_sa, const void* Sb, int64_t sb_stride, int64_t n,
                        float* x, cudaStream_t st, const DevInfo& di, int64_t cap, const SolveLayout& Lo,
                        int32_t* launches) {
  char* base = (char*)p->solve_buf;
  SolveLaunch L;
  L.wait_cycles = p->solve_wait_cycles;
  L.SA = SA;
  L.Sb = Sb;
  L.lda_sa = lda_sa;
  L.sb_stride = sb_stride;
  L.rule = p->rule;
  L.src_fp64 = 0;
  L.n = n;
  L.part = (double*)(base + Lo.part);
  L.bcast = (double*)(base + Lo.bcast);
  L.bar = (unsigned*)(base + Lo.bar);
  L.status = (unsigned*)(base + Lo.status);
  L.kappa = (double*)(base + Lo.kappa);
  L.x = x;
  // Tree levels: factor groups of at most `cap` rows, stack their [R | c] factors, repeat.
  int64_t rows = p->d;
  int level = 0;
  while (rows > cap) {
    const int64_t g = (rows + cap - 1) / cap;
    double* dst = (double*)(base + Lo.stack[level & 1]);
    const size_t es_src = L.src_fp64 ? sizeof(double) : elem_size(p->rule);
    for (int64_t gi = 0; gi < g; ++gi) {
      const int64_t r0 = gi * rows / g, r1 = (gi + 1) * rows / g;
      SolveLaunch G = L;
      G.SA = (const char*)L.SA + es_src * (size_t)(r0 * L.lda_sa);
      G.Sb = (const char*)L.Sb + es_src * (size_t)(r0 * L.sb_stride);
      G.d = r1 - r0;
      G.R = dst + gi * n * (n + 1);
      G.solve_x = 0;
      G.ncta = solve_ctas(G.d, n, di.sms, (size_t)di.optin);
      if (G.ncta < 1) return set_error(SK_ERR_UNSUPPORTED, "QR group of %lld rows does not fit", (long long)G.d);
      cudaError_t e = launch_solve(G, st, launches);
      if (e != cudaSuccess) return cuda_fail(e, "QR group launch");
    }
    L.SA = dst;
    L.Sb = dst + n;
    L.lda_sa = n + 1;
    L.sb_stride = n + 1;
    L.src_fp64 = 1;
    rows = g * n;
    ++level;
  }
  L.d = rows;
  L.R = (double*)(base + Lo.R);
  L.solve_x = 1;
  L.ncta = solve_ctas(rows, n, di.sms, (size_t)di.optin);
  if (L.ncta < 1) return set_error(SK_ERR_UNSUPPORTED, "FP64 QR of a %lld x %lld matrix does not fit", (long long)rows, (long long)(n + 1));
  cudaError_t e = launch_solve(L, st, launches);
  if (e != cudaSuccess) return cuda_fail(e, "QR launch");
  return SK_OK;
}

}  // namespace

sk_status sk_solve(sk_plan p, const float* A, int64_t lda, int64_t n, const float* b, float* x, void* stream) {
  clear_error();
  sk_status s = validate_apply(p, A, lda, n, x);
  if (s != SK_OK) return s;
  if (!b) return set_error(SK_ERR_INVALID_ARG, "b is NULL");
  if (n > p->d) return set_error(SK_ERR_INVALID_ARG, "sketch-and-solve needs n=%lld <= d=%lld", (long long)n, (long long)p->d);
  if (n > kMaxSolveN) return set_error(SK_ERR_UNSUPPORTED, "sketch-and-solve supports n <= %d", kMaxSolveN);
  DevInfo di;
  s = dev_info(&di);
  if (s != SK_OK) return s;
  const int64_t cap = solve_group_cap(p, n, di);
  if (cap < 1)
    return set_error(SK_ERR_UNSUPPORTED, "FP64 QR of a %lld x %lld sketch: too many columns for shared memory",
                     (long long)p->d, (long long)(n + 1));
  const int64_t groups1 = (p->d > cap) ? (p->d + cap - 1) / cap : 0;
  const SolveLayout Lo = solve_layout(p->d, n, p->rule, groups1);
  if (p->solve_bytes < Lo.total) {
    s = plan_grow(p, &p->solve_buf, &p->solve_bytes, Lo.total, "sketch-and-solve scratch");
    if (s != SK_OK) return s;
    // On the call's stream: a memset on the legacy default stream is not ordered with a non-blocking
    // caller stream and could land after this call's kernels have written the scratch.
    cudaError_t ez = cudaMemsetAsync(p->solve_buf, 0, Lo.total, (cudaStream_t)stream);
    if (ez != cudaSuccess) return cuda_fail(ez, "zeroing sketch-and-solve scratch");
  }
  p->solve_status_off = Lo.status;
  p->solve_kappa_off = Lo.kappa;
  char* base = (char*)p->solve_buf;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t launches = 0;
  const size_t es = elem_size(p->rule);
  cudaError_t e = cudaMemsetAsync(base + Lo.ya, 0, Lo.part - Lo.ya, st);  // Y_A and Y_b
  if (e != cudaSuccess) return cuda_fail(e, "zeroing sketches");
  e = cudaMemsetAsync(base + Lo.status, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing status");
  (void)es;
  int64_t R_used = 0;
  s = enqueue_sketch(p, A, lda, n, p->row_offset, p->m, base + Lo.ya, 0, st, &launches, &R_used);
  if (s != SK_OK) return s;
  // Sb is column n of [A | b]: the same chunks, and the rounding bits of global column n.
  s = enqueue_sketch(p, b, 1, 1, p->row_offset, p->m, base + Lo.yb, R_used, st, &launches, nullptr, n);
  if (s != SK_OK) return s;
  s = solve_backend(p, base + Lo.ya, n, base + Lo.yb, 1, n, x, st, di, cap, Lo, &launches);
  if (s != SK_OK) return s;
  p->last_launches = launches;
  p->last_R = R_used;
  return SK_OK;
}

sk_status sk_solve_sketched(sk_plan p, const void* SAb, int64_t ld, int64_t n, float* x, void* stream) {
  clear_error();
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  if (!SAb || !x) return set_error(SK_ERR_INVALID_ARG, "NULL sketch or x");
  if (n < 1 || ld < n + 1) return set_error(SK_ERR_INVALID_ARG, "need n >= 1 and ld >= n + 1 (n=%lld ld=%lld)",
                                            (long long)n, (long long)ld);
  if (n > p->d) return set_error(SK_ERR_INVALID_ARG, "sketch-and-solve needs n=%lld <= d=%lld", (long long)n, (long long)p->d);
  if (n > kMaxSolveN) return set_error(SK_ERR_UNSUPPORTED, "sketch-and-solve supports n <= %d", kMaxSolveN);
  const size_t es = elem_size(p->rule);
  if ((reinterpret_cast<uintptr_t>(SAb) % es) != 0) return set_error(SK_ERR_INVALID_ARG, "sketch not aligned to its elements");
  DevInfo di;
  sk_status s = dev_info(&di);
  if (s != SK_OK) return s;
  const int64_t cap = solve_group_cap(p, n, di);
  if (cap < 1)
    return set_error(SK_ERR_UNSUPPORTED, "FP64 QR of a %lld x %lld sketch: too many columns for shared memory",
                     (long long)p->d, (long long)(n + 1));
  const int64_t groups1 = (p->d > cap) ? (p->d + cap - 1) / cap : 0;
  const SolveLayout Lo = solve_layout(p->d, n, p->rule, groups1);
  if (p->solve_bytes < Lo.total) {
    s = plan_grow(p, &p->solve_buf, &p->solve_bytes, Lo.total, "sketch-and-solve scratch");
    if (s != SK_OK) return s;
    // On the call's stream: a memset on the legacy default stream is not ordered with a non-blocking
    // caller stream and could land after this call's kernels have written the scratch.
    cudaError_t ez = cudaMemsetAsync(p->solve_buf, 0, Lo.total, (cudaStream_t)stream);
    if (ez != cudaSuccess) return cuda_fail(ez, "zeroing sketch-and-solve scratch");
  }
  p->solve_status_off = Lo.status;
  p->solve_kappa_off = Lo.kappa;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync((char*)p->solve_buf + Lo.status, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing status");
  int32_t launches = 0;
  const char* sa = static_cast<const char*>(SAb);
  s = solve_backend(p, sa, ld, sa + es * (size_t)n, ld, n, x, st, di, cap, Lo, &launches);
  if (s != SK_OK) return s;
  p->last_launches = launches;
  return SK_OK;
}

sk_status sk_solve_precond(sk_plan p, const float* A, int64_t lda, int64_t n, const float* b, double* x,
                           int32_t max_iters, double tol, int32_t* iters_out, void* stream) {
  clear_error();
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  if (!x) return set_error(SK_ERR_INVALID_ARG, "x is NULL");
  if (n > kLsqrMaxN) return set_error(SK_ERR_UNSUPPORTED, "sketch-and-precondition supports n <= %d", kLsqrMaxN);
  if (max_iters <= 0) max_iters = 100;
  if (!(tol > 0.0)) tol = 1e-10;
  cudaStream_t st = (cudaStream_t)stream;
  // Scratch: u (m doubles), v w y p z x0 (6 n-vectors), scalars, the FP32 sketch-and-solve x0.
  const int64_t m = p->m;
  const size_t nv = (size_t)((n + 31) / 32 * 32);
  const size_t need = sizeof(double) * ((size_t)m + 6 * nv + kLsqrScalars) + sizeof(float) * nv;
  if (p->lsqr_bytes < need) {
    sk_status sg = plan_grow(p, &p->lsqr, &p->lsqr_bytes, need, "sketch-and-precondition scratch");
    if (sg != SK_OK) return sg;
  }
  double* base = p->lsqr;
  float* x0f = reinterpret_cast<float*>(base + m + 6 * nv + kLsqrScalars);
  sk_status s = sk_solve(p, A, lda, n, b, x0f, stream);
  if (s != SK_OK) return s;
  const int64_t solve_launches = p->last_launches;
  s = sk_solve_status(p, nullptr, stream);
  if (s != SK_OK) return s;
  DevInfo di;
  s = dev_info(&di);
  if (s != SK_OK) return s;
  LsqrLaunch L;
  L.A = A;
  L.lda = lda;
  L.m = m;
  L.n = n;
  const SolveLayout Lo = solve_layout(p->d, n, p->rule, 0);  // the offset of R does not depend on the tree
  L.R = reinterpret_cast<const double*>((char*)p->solve_buf + Lo.R);
  L.ldr = n + 1;
  L.u = base;
  L.v = base + m;
  L.w = L.v + nv;
  L.y = L.w + nv;
  L.p = L.y + nv;
  L.z = L.p + nv;
  L.x0 = L.z + nv;
  L.sc = L.x0 + nv;
  L.x = x;
  int32_t launches = (int32_t)solve_launches;
  cudaError_t e = lsqr_start(L, b, x0f, di.sms, st, &launches);
  if (e != cudaSuccess) return cuda_fail(e, "LSQR start");
  double sc[kLsqrScalars];
  int32_t it = 0;
  while (it < max_iters) {
    e = lsqr_iterate(L, di.sms, st, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "LSQR iteration");
    ++it;
    if (it % 4 != 0 && it != max_iters) continue;
    e = cudaMemcpyAsync(sc, L.sc, sizeof(sc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "LSQR convergence test");
    if (sc[kLsqrDone] != 0.0) break;
    const double anorm = sqrt(sc[kLsqrAnorm2]);
    const double rnorm = sc[kLsqrRnorm], arnorm = sc[kLsqrArnorm];
    if (!std::isfinite(rnorm) || !std::isfinite(arnorm))
      return set_error(SK_ERR_NUMERIC, "LSQR produced a non-finite residual estimate");
    if (rnorm <= tol * sc[kLsqrBnorm] || arnorm <= tol * anorm * rnorm) break;
  }
  e = lsqr_finish(L, st, &launches);
  if (e != cudaSuccess) return cuda_fail(e, "LSQR finish");
  e = cudaMemcpyAsync(sc, L.sc, sizeof(sc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "LSQR result");
  if (iters_out) *iters_out = (int32_t)sc[kLsqrIters];
  p->last_launches = launches;
  return SK_OK;
}

sk_status sk_apply_partials(sk_plan p, const float* A, int64_t lda, int64_t n, float* P, int64_t t0, int64_t nchunks,
                            void* stream) {
  clear_error();
  sk_status s = validate_apply(p, A, lda, n, P);
  if (s != SK_OK) return s;
  if ((reinterpret_cast<uintptr_t>(P) & 15u) != 0) return set_error(SK_ERR_INVALID_ARG, "P must be 16-byte aligned");
  if (p->mode != SK_MODE_ATOMIC || p->kernel == SK_KERNEL_LITERAL)
    return set_error(SK_ERR_UNSUPPORTED, "sk_apply_partials runs in atomic mode with a chunked kernel");
  const int64_t R = p->R;
  if (R <= 0)
    return set_error(SK_ERR_INVALID_ARG,
                     "sk_apply_partials needs SK_PARAM_CHUNK_ROWS set (the same on every shard of the matrix)");
  const int64_t tf = p->row_offset / R, tl = (p->row_offset + p->m - 1) / R;
  if (t0 < 0 || nchunks < 1 || tf < t0 || tl >= t0 + nchunks)
    return set_error(SK_ERR_INVALID_ARG, "the plan's chunks [%lld, %lld] are not inside P's chunks [%lld, %lld)",
                     (long long)tf, (long long)tl, (long long)t0, (long long)(t0 + nchunks));
  DevInfo di;
  s = dev_info(&di);
  if (s != SK_OK) return s;
  TileCfg cfg;
  s = choose_tile(p, n, p->m, di, &cfg, tma_layout_ok(A, lda), true);
  if (s != SK_OK) return s;
  if (cfg.glob) {
    // The global kernel finishes its passes as it goes; partials take the tile kernel instead.
    sk_plan_s tmp = *p;
    tmp.kernel = SK_KERNEL_TILE;
    s = choose_tile(&tmp, n, p->m, di, &cfg, tma_layout_ok(A, lda), true);
    if (s != SK_OK) return s;
  }
  cfg.R = R;
  if (!cfg.reg && cfg.slices < 2) cfg.slices = 2;  // work items flush into the chunk totals
  if (!p->dstatus) {
    size_t cur = 0;
    s = plan_grow(p, &p->dstatus, &cur, sizeof(unsigned), "status word");
    if (s != SK_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(p->dstatus, 0, sizeof(unsigned), st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "zeroing status");
  TileLaunch L;
  L.A = A;
  L.a_type = SK_A_FP32;
  L.Y = nullptr;
  L.lda = lda;
  L.n = n;
  L.row_begin = p->row_offset;
  L.row_end = p->row_offset + p->m;
  L.d = p->d;
  L.k = p->k;
  L.rule = p->rule;
  L.seed = p->seed;
  L.scale = p->scale;
  L.R = R;
  L.NC = cfg.NC;
  L.kb = cfg.kb;
  L.threads = cfg.threads;
  L.grid = cfg.grid;
  L.slices = cfg.slices;
  L.depth = cfg.depth;
  L.mb = cfg.mb;
  L.lr = cfg.lr ? 1 : 0;
  L.own = cfg.own ? 1 : 0;
  L.vec = cfg.vec ? 1 : 0;
  L.glob = 0;
  L.reg = cfg.reg ? 1 : 0;
  L.reg_nsub = cfg.reg_nsub;
  L.reg_cap = cfg.reg_cap;
  L.col_off = 0;
  L.allow_tma = cfg.vec ? 0 : 1;
  L.status = p->dstatus;
  L.P = P + (tf - t0) * p->d * n;
  L.no_finish = 1;
  int32_t launches = 0;
  cudaError_t e = launch_tile(L, st, &launches);
  if (e != cudaSuccess) return cuda_fail(e, "sketch kernel launch (partials)");
  p->last_noalloc = false;
  p->last_launches = launches;
  p->last_R = R;
  p->last_kernel = cfg.reg ? SK_KERNEL_REGISTER : cfg.own ? SK_KERNEL_OWNER : SK_KERNEL_TILE;
  return SK_OK;
}

sk_status sk_finish_partials(sk_plan p, float* P, int64_t t0, int64_t nchunks, int64_t n, void* Y, void* stream) {
  clear_error();
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  if (!P || !Y) return set_error(SK_ERR_INVALID_ARG, "P and Y must not be NULL");
  if (n < 1 || n > kMaxN) return set_error(SK_ERR_INVALID_ARG, "n=%lld outside [1, %lld]", (long long)n, (long long)kMaxN);
  if (t0 < 0 || nchunks < 1) return set_error(SK_ERR_INVALID_ARG, "need t0 >= 0 and nchunks >= 1");
  if ((reinterpret_cast<uintptr_t>(P) & 15u) != 0) return set_error(SK_ERR_INVALID_ARG, "P must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(Y) & 3u) != 0) return set_error(SK_ERR_INVALID_ARG, "Y must be 4-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(Y, 0, elem_size(p->rule) * (size_t)(p->d * n), st);
  if (e != cudaSuccess) return cuda_fail(e, "zeroing Y");
  TileDesc D;
  memset(&D, 0, sizeof(D));
  D.Y = Y;
  D.n = n;
  D.seed = p->seed;
  D.scale = p->scale;
  D.B = (uint32_t)p->B;
  D.k = (uint32_t)p->k;
  D.kp = (uint32_t)((p->k + 1) / 2);
  D.col_off = 0;
  D.ldy = 0;
  int32_t launches = 0;
  e = launch_chunk_finish(D, p->rule, P, t0, nchunks, st, &launches);
  if (e != cudaSuccess) return cuda_fail(e, "chunk-finish launch");
  p->last_launches = launches;
  return SK_OK;
}

sk_status sk_solve_status(sk_plan p, double* kappa, void* stream) {
  clear_error();
  if (!p) return set_error(SK_ERR_INVALID_ARG, "plan is NULL");
  if (!p->solve_buf) return set_error(SK_ERR_INVALID_ARG, "no sk_solve has run on this plan");
  cudaStream_t st = (cudaStream_t)stream;
  // One copy of the status word and kappa (adjacent in the scratch layout), ordered on the caller's
  // stream: a copy on the legacy default stream would also wait for unrelated work queued there.
  unsigned status = 0;
  double kap = 0.0;
  const size_t lo = std::min(p->solve_status_off, p->solve_kappa_off);
  const size_t hi = std::max(p->solve_status_off + 4, p->solve_kappa_off + 8);
  unsigned char words[1024];
  cudaError_t e;
  if (hi - lo <= sizeof(words)) {
    e = cudaMemcpyAsync(words, (char*)p->solve_buf + lo, hi - lo, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading solve status");
    memcpy(&status, words + (p->solve_status_off - lo), 4);
    memcpy(&kap, words + (p->solve_kappa_off - lo), 8);
  } else {
    e = cudaMemcpyAsync(&status, (char*)p->solve_buf + p->solve_status_off, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kap, (char*)p->solve_buf + p->solve_kappa_off, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading solve status");
  }
  if (kappa) *kappa = kap;
  if (status & 1u) return set_error(SK_ERR_TIMEOUT, "a grid barrier of the QR kernel timed out");
  if (status & 2u) return set_error(SK_ERR_NUMERIC, "SA is rank deficient (zero pivot in the QR)");
  return SK_OK;
}

void sk_destroy(sk_plan p) {
  if (!p) return;
  cudaDeviceSynchronize();
  if (p->det_P) cudaFree(p->det_P);
  if (p->dstatus) cudaFree(p->dstatus);
  if (p->tileP) cudaFree(p->tileP);
  if (p->lsqr) cudaFree(p->lsqr);
  if (p->solve_buf) cudaFree(p->solve_buf);
  for (int b = 0; b < 2; ++b) {
    if (p->stage[b]) cudaFree(p->stage[b]);
    if (p->ev_copied[b]) cudaEventDestroy(p->ev_copied[b]);
    if (p->ev_used[b]) cudaEventDestroy(p->ev_used[b]);
  }
  if (p->ydev) cudaFree(p->ydev);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  delete p;
}

}  // extern "C"

namespace sk {

// Tile-kernel launch description for sk_apply_noalloc (sk_noalloc.cu): the same configuration
// sk_apply's atomic tile path chooses, with no scratch attached. Allocates nothing.
sk_status noalloc_tile_launch(const sk_plan_s* p, const float* A, int64_t lda, int64_t n, void* Y, TileLaunch* L) {
  sk_status s = validate_apply(p, A, lda, n, Y);
  if (s != SK_OK) return s;
  if (p->mode != SK_MODE_ATOMIC || p->kernel == SK_KERNEL_LITERAL)
    return set_error(SK_ERR_UNSUPPORTED, "sk_apply_noalloc runs the atomic-mode tile kernel only");
  DevInfo di;
  s = dev_info(&di);
  if (s != SK_OK) return s;
  TileCfg cfg;
  s = choose_tile(p, n, p->m, di, &cfg, tma_layout_ok(A, lda));
  if (s != SK_OK) return s;
  L->A = A;
  L->Y = Y;
  L->lda = lda;
  L->n = n;
  L->row_begin = p->row_offset;
  L->row_end = p->row_offset + p->m;
  L->d = p->d;
  L->k = p->k;
  L->rule = p->rule;
  L->seed = p->seed;
  L->scale = p->scale;
  L->R = cfg.R;
  L->NC = cfg.NC;
  L->kb = cfg.kb;
  L->threads = cfg.threads;
  L->grid = cfg.grid;
  L->slices = cfg.slices;
  L->depth = cfg.depth;
  L->mb = cfg.mb;
  L->lr = cfg.lr ? 1 : 0;
  L->own = cfg.own ? 1 : 0;
  L->vec = cfg.vec ? 1 : 0;
  L->glob = cfg.glob ? 1 : 0;
  L->reg = cfg.reg ? 1 : 0;
  L->reg_nsub = cfg.reg_nsub;
  L->reg_cap = cfg.reg_cap;
  L->col_off = 0;
  L->allow_tma = 1;
  L->status = nullptr;
  L->P = nullptr;
  return SK_OK;
}

size_t noalloc_elem_size(const sk_plan_s* p) { return elem_size(p->rule); }

void noalloc_record(sk_plan_s* p, int64_t launches, int64_t R, int32_t kernel) {
  p->last_launches = launches;
  p->last_R = R;
  p->last_kernel = kernel;
  p->last_noalloc = true;
}

}  // namespace sk
