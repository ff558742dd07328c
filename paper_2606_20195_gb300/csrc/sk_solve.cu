// FP64 back end of sketch-and-solve least squares (paper Sec. 5.1: minimize ||SA x - Sb||_2 through
// a reduced QR of SA and a triangular solve). The paper factors in FP32; here the factorization,
// Q^T Sb and the back substitution run in FP64.
//
// One cooperative launch factors W = [SA | Sb] (d x (n+1)) by Householder reflections. The d rows
// are split across the CTAs (one per SM at most); each CTA keeps its rows of W in shared memory
// for the whole factorization. A sketch too tall for the GPU's shared memory is factored as a tree
// (TSQR): groups of rows are factored by separate launches, their n x (n+1) factors [R_g | c_g] are
// stacked in FP64 and factored again, until one launch holds the whole stack. Dropping each group's
// last row (its residual norm) only removes a constant from ||W x~||, so the minimizer is unchanged. Column step j needs one grid-wide reduction: the partial sums of
// x^T x and x^T W[:, c] (x = column j below the diagonal) give both the reflector and v^T W[:, c],
// accumulated with FP64 atomics into per-step buffers, followed by one grid synchronization. The owner of row j
// publishes that row before the barrier; after the last step every owner writes its final rows of R
// and CTA 0 finishes with the back substitution R x = (Q^T Sb)[:n].
//
// Every grid synchronization waits at most about two seconds: on expiry the kernel sets
// kStatusTimeout in the status word and all CTAs leave at the next check, so a stalled launch cannot
// hang the GPU.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "sk_device.cuh"
#include "sk_internal.h"

namespace sk {

namespace {

// Columns of W = [SA | Sb] the kernel handles (n + 1 <= kQRMaxCols), and per thread of a 256-thread
// CTA in one column step.
constexpr int kQRMaxCols = 1032;
constexpr int kQRThreads = 256;
constexpr int kQRColsPerThread = (kQRMaxCols + kQRThreads - 1) / kQRThreads;

// A grid barrier gives up after about two seconds of waiting (in SM clock cycles at ~2 GHz).
constexpr long long kBarrierCycles = 4000000000ll;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid synchronization for a co-resident (cooperative) grid with monotonic arrival counters (zero at
// launch and never reset): every CTA's thread 0 adds 1 with release semantics, after a CTA barrier,
// to counter b mod kBarCounters (128 bytes apart), then polls them with acquire loads until their sum
// reaches `target` (= grid size x synchronization number). The CTA's writes before the call are
// visible to every CTA after it. Gives up after `limit` SM clock cycles. Returns false if this CTA, or
// any CTA before it, gave up waiting.
// One counter: spreading the arrivals over 8 counters was measured slower on GB300 (QR at n = 1024,
// d = 2048: 12.7 -> 14.6 ms), the polls of 8 counters costing more than the queued arrivals.
constexpr int kBarCounters = 1;
constexpr int kBarStride = 32;  // unsigned words between counters

__device__ bool grid_arrive_wait(unsigned* bar, unsigned target, unsigned* status, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* mine = bar + (blockIdx.x % kBarCounters) * kBarStride;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(mine) : "memory");
    const long long t0 = clock64();
    unsigned polls = 0;
    while (true) {
      unsigned sum = 0;
#pragma unroll
      for (int q = 0; q < kBarCounters; ++q) sum += ld_acquire_u32(bar + q * kBarStride);
      if (sum >= target) break;
      // the clock is read on the first poll (so that a limit of a few cycles takes effect at once)
      // and every 256 polls after it
      if ((++polls & 255u) == 1u || (polls & 255u) == 0u) {
        if (clock64() - t0 > limit) {
          atomicOr(status, kStatusTimeout);
          break;
        }
        // Another CTA already gave up: stop waiting.
        if (*(volatile unsigned*)status & kStatusTimeout) break;
      }
      if (polls > 512) __nanosleep(32);
    }
    ok = (*(volatile unsigned*)status & kStatusTimeout) == 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct QRArgs {
  SolveLaunch L;
  int32_t rpc;     // rows per CTA
  double* nrm;     // n doubles, zeroed
  double* wv;      // n * (n+1) doubles, zeroed
};

template <typename T>
__device__ __forceinline__ double load_val(const void* p, int64_t idx) {
  if constexpr (std::is_same<T, double>::value) return reinterpret_cast<const double*>(p)[idx];
  else if constexpr (std::is_same<T, __half>::value) return (double)__half2float(reinterpret_cast<const __half*>(p)[idx]);
  else if constexpr (std::is_same<T, __nv_bfloat16>::value)
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
  else return (double)reinterpret_cast<const float*>(p)[idx];
}

// Columns c > j + 1 of this CTA's rows r >= j: apply step j's reflector (W[r][c] -= tv_r w_c, with
// tv_r = tau v_r staged per row; tv = 0 before the first step) and accumulate the next step's partial
// sums x^T W[:, c] over rows r >= j + 1 (x_r = W[r][j+1] after the update, 0 on row j). Four columns
// per thread at a time (independent chains), rows in the inner loop; one atomic per column.
__device__ __forceinline__ void qr_sweep(double* Wl, int64_t ldw, int64_t n, int64_t j, int64_t rl0, int64_t nown,
                                         const double* tvs, const double* xns, const double* wsm, bool update,
                                         double* wv_next) {
  const int64_t jn = j + 1;
  for (int64_t cb = jn + 1 + threadIdx.x; cb <= n; cb += 4 * (int64_t)blockDim.x) {
    double dot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t rl = rl0; rl < nown; ++rl) {
      double* wrow = Wl + rl * ldw;
      const double tv = tvs[rl], xv = xns[rl];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t c = cb + q * (int64_t)blockDim.x;
        if (c <= n) {
          double w = wrow[c];
          if (update) {
            w -= tv * wsm[c];
            wrow[c] = w;
          }
          dot[q] += xv * w;
        }
      }
    }
    if (wv_next) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t c = cb + q * (int64_t)blockDim.x;
        if (c <= n && dot[q] != 0.0) atomicAdd(&wv_next[c], dot[q]);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kQRThreads) qr64_kernel(const QRArgs a) {
  const long long wait = a.L.wait_cycles > 0 ? a.L.wait_cycles : kBarrierCycles;
  // rpc x (n+1) rows of W (row-major), then tv_r and the next column's x_r for each local row
  extern __shared__ __align__(16) double Wl[];
  __shared__ double sc[4];
  __shared__ double wsm[kQRMaxCols];  // w_c = v^T W[:, c] of the current column step
  const SolveLaunch& L = a.L;
  const int64_t n = L.n, d = L.d, ldw = n + 1;
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const unsigned nb = gridDim.x;
  const int64_t row0 = (int64_t)b * a.rpc;
  const int64_t nown = max((int64_t)0, min((int64_t)a.rpc, d - row0));
  double* tvs = Wl + (int64_t)a.rpc * ldw;
  double* xns = tvs + a.rpc;
  // Load own rows of [SA | Sb] as FP64.
  for (int64_t e = threadIdx.x; e < nown * ldw; e += blockDim.x) {
    const int64_t rl = e / ldw, c = e - rl * ldw;
    const int64_t r = row0 + rl;
    Wl[e] = (c < n) ? load_val<T>(L.SA, r * L.lda_sa + c) : load_val<T>(L.Sb, r * L.sb_stride);
  }
  __syncthreads();
  // One grid reduction per column: with x = W[j:, j] and v = x - alpha e_j, both ||x||^2 and
  // v^T W[:, c] = x^T W[:, c] - alpha W[j][c] follow from the partial sums of x^T x and x^T W[:, c]
  // over each CTA's rows; the owner of row j publishes that row. Step j's update of the trailing
  // columns and the partial sums of step j + 1 share one pass over the rows (qr_sweep).
  {
    double ss = 0.0;
    for (int64_t rl = threadIdx.x; rl < nown; rl += blockDim.x) {
      const double x = Wl[rl * ldw];
      tvs[rl] = 0.0;
      xns[rl] = x;
      ss += x * x;
    }
    ss = warp_sum(ss);
    if (lane == 0 && ss != 0.0) atomicAdd(&a.nrm[0], ss);
    __syncthreads();
    qr_sweep(Wl, ldw, n, -1, 0, nown, tvs, xns, wsm, false, a.wv);
    if (row0 == 0 && nown > 0)
      for (int64_t c = threadIdx.x; c <= n; c += blockDim.x) L.R[c] = Wl[c];
  }
  if (!grid_arrive_wait(L.bar, nb, L.status, wait)) return;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t jn = j + 1;
    // Inputs of w_c = x^T W[:, c] - alpha W[j][c] for this thread's columns c > j, loaded while
    // thread 0 forms the reflector (kQRColsPerThread columns per thread at 256 threads).
    double wraw[kQRColsPerThread], rraw[kQRColsPerThread];
#pragma unroll
    for (int q = 0; q < kQRColsPerThread; ++q) {
      const int64_t c = jn + threadIdx.x + q * (int64_t)blockDim.x;
      wraw[q] = (c <= n) ? __ldcg(&a.wv[j * ldw + c]) : 0.0;
      rraw[q] = (c <= n) ? __ldcg(&L.R[j * ldw + c]) : 0.0;
    }
    const double wn_raw = (jn <= n) ? __ldcg(&a.wv[j * ldw + jn]) : 0.0;
    const double rn_raw = (jn <= n) ? __ldcg(&L.R[j * ldw + jn]) : 0.0;
    // Reflector, formed once per CTA (FP64 square root and division are long instruction sequences
    // on this part's FP64 pipe): alpha = -sign(x0) ||x||, v_j = x0 - alpha, tau = 2 / v^T v.
    if (threadIdx.x == 0) {
      const double norm2 = __ldcg(&a.nrm[j]);
      const double x0 = __ldcg(&L.R[j * ldw + j]);
      const double al = -copysign(sqrt(norm2), x0);
      const double v0 = x0 - al;
      const double vtv = (norm2 - x0 * x0) + v0 * v0;
      sc[0] = al;
      sc[1] = v0;
      sc[2] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    }
    __syncthreads();
    const double alpha = sc[0], vj = sc[1], tau = sc[2];
    // w_c for c > j, staged once per CTA; the rows' own threads use the same expression for
    // column j + 1.
#pragma unroll
    for (int q = 0; q < kQRColsPerThread; ++q) {
      const int64_t c = jn + threadIdx.x + q * (int64_t)blockDim.x;
      if (c <= n) wsm[c] = wraw[q] - alpha * rraw[q];
    }
    const double w_next = (jn <= n) ? wn_raw - alpha * rn_raw : 0.0;
    // Per row r >= j: tv_r = tau v_r, column j + 1 updated (the next step's x_r), the row's share
    // of ||x||^2 for step j + 1; the owner's diagonal becomes alpha.
    const int64_t rl0 = max((int64_t)0, min(nown, j - row0));  // first local row with r >= j
    double ss = 0.0;
    for (int64_t rl = rl0 + threadIdx.x; rl < nown; rl += blockDim.x) {
      const int64_t r = row0 + rl;
      double* wrow = Wl + rl * ldw;
      const double tv = tau * ((r == j) ? vj : wrow[j]);
      tvs[rl] = tv;
      double xn = 0.0;
      if (jn <= n) {
        xn = wrow[jn] - tv * w_next;
        wrow[jn] = xn;
      }
      xns[rl] = (r >= jn) ? xn : 0.0;
      if (r >= jn) ss += xn * xn;
      if (r == j) wrow[j] = alpha;
    }
    ss = warp_sum(ss);
    if (jn < n && lane == 0 && ss != 0.0) atomicAdd(&a.nrm[jn], ss);
    __syncthreads();
    qr_sweep(Wl, ldw, n, j, rl0, nown, tvs, xns, wsm, tau != 0.0, (jn < n) ? a.wv + jn * ldw : nullptr);
    if (jn < n) {
      __syncthreads();
      if (jn >= row0 && jn < row0 + nown) {
        const int64_t rl = jn - row0;
        for (int64_t c = jn + threadIdx.x; c <= n; c += blockDim.x) L.R[jn * ldw + c] = Wl[rl * ldw + c];
      }
      if (!grid_arrive_wait(L.bar, nb * (unsigned)(jn + 1), L.status, wait)) return;
    }
  }
  // Final R rows: each owner rewrites its rows of R (diagonal alpha, updated off-diagonals).
  if (!grid_arrive_wait(L.bar, nb * (unsigned)(n + 1), L.status, wait)) return;
  for (int64_t jr = row0; jr < row0 + nown && jr < n; ++jr) {
    const int64_t rl = jr - row0;
    for (int64_t c = jr + threadIdx.x; c <= n; c += blockDim.x) L.R[jr * ldw + c] = Wl[rl * ldw + c];
  }
  // A group of a tree level: the rows of [R | c] are its whole output (below the diagonal stays 0).
  if (!L.solve_x) {
    for (int64_t jr = row0; jr < row0 + nown && jr < n; ++jr)
      for (int64_t c = threadIdx.x; c < jr; c += blockDim.x) L.R[jr * ldw + c] = 0.0;
    return;
  }
  if (!grid_arrive_wait(L.bar, nb * (unsigned)(n + 2), L.status, wait)) return;
  if (b != 0) return;
  // Back substitution on CTA 0 (column-oriented): rhs in shared memory (reuses Wl).
  double* rhs = Wl;
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) rhs[l] = __ldcg(&L.R[l * ldw + n]);
  __syncthreads();
  double rmax = 0.0, rmin = 0.0;
  bool singular = false;
  for (int64_t j = n - 1; j >= 0; --j) {
    const double rjj = __ldcg(&L.R[j * ldw + j]);
    if (threadIdx.x == 0) {
      const double xj = (rjj != 0.0) ? rhs[j] / rjj : 0.0;
      rhs[j] = xj;
      sc[3] = xj;
    }
    if (rjj == 0.0) singular = true;
    const double arj = fabs(rjj);
    if (j == n - 1) {
      rmax = arj;
      rmin = arj;
    } else {
      rmax = fmax(rmax, arj);
      rmin = fmin(rmin, arj);
    }
    __syncthreads();
    const double xj = sc[3];
    for (int64_t l = threadIdx.x; l < j; l += blockDim.x) rhs[l] -= __ldcg(&L.R[l * ldw + j]) * xj;
    __syncthreads();
  }
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) L.x[l] = singular ? __int_as_float(0x7fc00000) : (float)rhs[l];
  if (threadIdx.x == 0) {
    if (singular) atomicOr(L.status, kStatusNumeric);
    *L.kappa = (rmin > 0.0) ? rmax / rmin : __longlong_as_double(0x7ff0000000000000ll);
  }
}

// Dynamic shared memory a QR CTA may use: the opt-in limit less the static arrays and a margin.
size_t solve_smem_budget(size_t smem_optin) {
  const size_t fixed = sizeof(double) * (kQRMaxCols + 4) + 2048;
  return smem_optin > fixed ? smem_optin - fixed : 0;
}

}  // namespace

size_t solve_bar_bytes() { return sizeof(unsigned) * kBarCounters * kBarStride; }

int64_t solve_rows_cap(int64_t n, int32_t sms, size_t smem_optin) {
  if (n < 1 || n + 1 > kQRMaxCols) return 0;
  return (int64_t)sms * (int64_t)(solve_smem_budget(smem_optin) / ((size_t)(n + 3) * 8));
}

int32_t solve_ctas(int64_t d, int64_t n, int32_t sms, size_t smem_optin) {
  if (n < 1 || d < n || n + 1 > kQRMaxCols) return 0;
  const size_t budget = solve_smem_budget(smem_optin);
  int64_t ncta = std::min<int64_t>(sms, std::max<int64_t>(1, (d + 7) / 8));
  for (; ncta <= sms; ++ncta) {
    const int64_t rpc = (d + ncta - 1) / ncta;
    if ((size_t)rpc * (size_t)(n + 3) * 8 <= budget) return (int32_t)ncta;
  }
  return 0;
}

cudaError_t launch_solve(const SolveLaunch& L, cudaStream_t st, int32_t* launches) {
  QRArgs a;
  a.L = L;
  a.rpc = (int32_t)((L.d + L.ncta - 1) / L.ncta);
  // part scratch holds nrm (n) followed by wv (n * (n+1)).
  a.nrm = L.part;
  a.wv = L.part + L.n;
  cudaError_t e = cudaMemsetAsync(L.part, 0, sizeof(double) * (size_t)(L.n + L.n * (L.n + 1)), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.bar, 0, solve_bar_bytes(), st);
  if (e != cudaSuccess) return e;
  const size_t smem = std::max<size_t>((size_t)a.rpc * (size_t)(L.n + 3) * 8, (size_t)L.n * 8);
  void* args[] = {(void*)&a};
  const void* kern = L.src_fp64          ? (const void*)qr64_kernel<double>
                     : (L.rule == kFP32) ? (const void*)qr64_kernel<float>
                     : (L.rule == kBF16) ? (const void*)qr64_kernel<__nv_bfloat16>
                                         : (const void*)qr64_kernel<__half>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)L.ncta), dim3(kQRThreads), args, smem, st);
  if (launches) *launches += 1;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sk
