// Sketch-and-precondition least squares: LSQR (Paige and Saunders, ACM TOMS 1982) on A with the
// right preconditioner R^{-1}, where S A = Q R is the FP64 QR of the sketch from sk_solve (paper
// Sec. 5.1 forms S A and its QR; the discussion names sketch-and-precondition as the use of that R
// as a preconditioner). The preconditioned operator M = A R^{-1} has singular values within the
// sketch's distortion of 1, so LSQR needs few iterations, and it converges to the least-squares
// solution of A itself: the rounding rule of the sketch only changes the preconditioner.
//
// Everything of an iteration runs on the GPU. The two products with A run on the FP32 pipe with
// about twice FP32 precision (exact products and compensated sums, df_acc); vector lengths, the
// step and the recurrence are FP64:
//   lsqr_av_kernel    u <- A p - c u and ||u||^2           (one lane per row of A)
//   lsqr_atu_kernel   z <- A^T u                           (warps over row runs, FP64 atomics)
//   lsqr_step_kernel  the n-vector part: v = R^{-T} z / beta - beta v, alpha, the plane rotation,
//                     y and w updates, p = R^{-1} v        (one CTA; n <= 512)
// u is kept unnormalized (its scale is folded into the next step), the iterate is x = x0 + R^{-1} y
// with x0 the sketch-and-solve solution.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sk_device.cuh"
#include "sk_internal.h"

namespace sk {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of v into *out with one FP64 atomic (blockDim a multiple of 32, at most 1024).
__device__ void block_atomic_sum(double v, double* out) {
  __shared__ double part[32];
  v = warp_sum_d(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0.0;
    s = warp_sum_d(s);
    if (lane == 0 && s != 0.0) atomicAdd(out, s);
  }
  __syncthreads();
}

// Products of A's FP32 entries with an FP64 vector y = yh + yl (two floats) accumulated in about
// twice FP32 precision on the FP32 pipe: the product a * yh is split exactly into p + e (FMA), the
// running sum takes p through TwoSum (Knuth), and the error terms e + a * yl and the TwoSum errors are
// summed in a second float (cascaded summation, Ogita, Rump and Oishi, SIAM J. Sci. Comput. 2005).
// Explicit round-to-nearest intrinsics keep the compiler from fusing the error-free steps.
__device__ __forceinline__ void df_acc(float a, float yh, float yl, float& s, float& c) {
  const float p = __fmul_rn(a, yh);
  const float e = __fmaf_rn(a, yh, -p);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, __fmaf_rn(a, yl, e)));
}

__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// u_i <- A_i . p + c u_i with c = sc[kLsqrC] (or b_i - A_i . p when `b` is given),
// sc[kLsqrBeta2] += sum of u_i^2. One lane per row; p in shared memory as (hi, lo) floats; u is
// kept as (hi, lo) floats (uh = first m, ul = next m floats of the u buffer).
__global__ void __launch_bounds__(256) lsqr_av_kernel(const LsqrLaunch L, const float* b) {
  extern __shared__ float pf[];  // [0, n): hi, [n, 2n): lo
  const int64_t n = L.n;
  const double c = b ? 0.0 : L.sc[kLsqrC];
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) split_df(L.p[j], pf[j], pf[n + j]);
  __syncthreads();
  float* uh = reinterpret_cast<float*>(L.u);
  float* ul = uh + L.m;
  const bool vec = (n & 3) == 0 && (L.lda & 3) == 0 && (reinterpret_cast<uintptr_t>(L.A) & 15u) == 0;
  double sq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.m; i += (int64_t)gridDim.x * blockDim.x) {
    const float* a = L.A + i * L.lda;
    float s = 0.f, cc = 0.f;
    if (vec) {
      for (int64_t j = 0; j < n; j += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(a + j));
        df_acc(v.x, pf[j], pf[n + j], s, cc);
        df_acc(v.y, pf[j + 1], pf[n + j + 1], s, cc);
        df_acc(v.z, pf[j + 2], pf[n + j + 2], s, cc);
        df_acc(v.w, pf[j + 3], pf[n + j + 3], s, cc);
      }
    } else {
      for (int64_t j = 0; j < n; ++j) df_acc(__ldg(a + j), pf[j], pf[n + j], s, cc);
    }
    const double dot = (double)s + (double)cc;
    const double u = b ? ((double)b[i] - dot) : fma(c, (double)uh[i] + (double)ul[i], dot);
    float h, l;
    split_df(u, h, l);
    uh[i] = h;
    ul[i] = l;
    sq = fma(u, u, sq);
  }
  block_atomic_sum(sq, L.sc + kLsqrBeta2);
}

// z <- z + A^T u over this CTA's rows (z zero before the launch). Each warp takes a contiguous run of
// rows; lane l keeps the partial sums of columns l, l + 32, ... (NPL of them, NPL * 32 >= n) as
// (s, c) float pairs, 4 rows per step; the CTA's warps combine their sums in FP64 in shared memory and
// add them with FP64 atomics.
template <int NPL>
__global__ void __launch_bounds__(256) lsqr_atu_kernel(const LsqrLaunch L) {
  __shared__ double zs[8][NPL * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float sh[NPL], cl[NPL];
#pragma unroll
  for (int q = 0; q < NPL; ++q) sh[q] = cl[q] = 0.f;
  const float* uh = reinterpret_cast<const float*>(L.u);
  const float* ul = uh + L.m;
  const int64_t nwt = (int64_t)gridDim.x * 8;
  const int64_t wg = (int64_t)blockIdx.x * 8 + warp;
  const int64_t rows_per = (L.m + nwt - 1) / nwt;
  const int64_t r0 = wg * rows_per;
  const int64_t r1 = min(L.m, r0 + rows_per);
  int64_t i = r0;
  for (; i + 4 <= r1; i += 4) {
    float h[4], l[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      h[t] = uh[i + t];
      l[t] = ul[i + t];
    }
    const float* a = L.A + i * L.lda;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int64_t j = lane + 32 * q;
      if (j < L.n) {
        float av[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) av[t] = __ldg(a + t * L.lda + j);
#pragma unroll
        for (int t = 0; t < 4; ++t) df_acc(av[t], h[t], l[t], sh[q], cl[q]);
      }
    }
  }
  for (; i < r1; ++i) {
    const float h = uh[i], l = ul[i];
    const float* a = L.A + i * L.lda;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int64_t j = lane + 32 * q;
      if (j < L.n) df_acc(__ldg(a + j), h, l, sh[q], cl[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NPL; ++q) zs[warp][lane + 32 * q] = (double)sh[q] + (double)cl[q];
  __syncthreads();
  for (int64_t j = threadIdx.x; j < L.n; j += blockDim.x) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += zs[w][j];
    if (t != 0.0) atomicAdd(L.z + j, t);
  }
}

// out = R^{-T} rhs (forward substitution on R^T, R upper triangular with row stride ldr), one CTA.
__device__ void solve_rt(const double* R, int64_t ldr, int64_t n, double* rhs) {
  for (int64_t i = 0; i < n; ++i) {
    __syncthreads();
    const double qi = rhs[i] / R[i * ldr + i];
    __syncthreads();
    if (threadIdx.x == 0) rhs[i] = qi;
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) rhs[j] = fma(-R[i * ldr + j], qi, rhs[j]);
  }
  __syncthreads();
}

// out = R^{-1} rhs (back substitution, column oriented), one CTA.
__device__ void solve_r(const double* R, int64_t ldr, int64_t n, double* rhs) {
  for (int64_t i = n - 1; i >= 0; --i) {
    __syncthreads();
    const double qi = rhs[i] / R[i * ldr + i];
    __syncthreads();
    if (threadIdx.x == 0) rhs[i] = qi;
    for (int64_t j = threadIdx.x; j < i; j += blockDim.x) rhs[j] = fma(-R[j * ldr + i], qi, rhs[j]);
  }
  __syncthreads();
}

__device__ double block_sum_sq(const double* x, int64_t n) {
  __shared__ double part[32];
  __shared__ double total;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s = fma(x[j], x[j], s);
  s = warp_sum_d(s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) part[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    total = t;
  }
  __syncthreads();
  return total;
}

// The n-vector part of an LSQR iteration (first: the initialization from r0 = b - A x0).
__global__ void __launch_bounds__(512) lsqr_step_kernel(const LsqrLaunch L, int first) {
  __shared__ double sh[kLsqrMaxN];
  const int64_t n = L.n;
  double* sc = L.sc;
  if (sc[kLsqrDone] != 0.0) return;
  const double beta = sqrt(sc[kLsqrBeta2]);
  // q = R^{-T} (A^T u_stored) / beta = M^T u (u normalized)
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) sh[j] = (beta > 0.0) ? L.z[j] / beta : 0.0;
  solve_rt(L.R, L.ldr, n, sh);
  if (!first)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) sh[j] = fma(-beta, L.v[j], sh[j]);
  const double alpha = sqrt(block_sum_sq(sh, n));
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) L.v[j] = (alpha > 0.0) ? sh[j] / alpha : 0.0;
  __syncthreads();
  if (first) {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      L.w[j] = L.v[j];
      L.y[j] = 0.0;
    }
    if (threadIdx.x == 0) {
      sc[kLsqrPhibar] = beta;
      sc[kLsqrRhobar] = alpha;
      sc[kLsqrAnorm2] = alpha * alpha;
      sc[kLsqrBnorm] = beta;
      sc[kLsqrRnorm] = beta;
      sc[kLsqrArnorm] = alpha * beta;
    }
  } else {
    const double rhobar = sc[kLsqrRhobar], phibar = sc[kLsqrPhibar];
    const double rho = hypot(rhobar, beta);
    const double cs = rhobar / rho, sn = beta / rho;
    const double theta = sn * alpha;
    const double phi = cs * phibar;
    const double t1 = phi / rho, t2 = -theta / rho;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double wj = L.w[j];
      L.y[j] = fma(t1, wj, L.y[j]);
      L.w[j] = fma(t2, wj, L.v[j]);
    }
    if (threadIdx.x == 0) {
      sc[kLsqrRhobar] = -cs * alpha;
      sc[kLsqrPhibar] = sn * phibar;
      sc[kLsqrAnorm2] += alpha * alpha + beta * beta;
      sc[kLsqrRnorm] = sn * phibar;
      sc[kLsqrArnorm] = sn * phibar * alpha * fabs(cs);
    }
  }
  // next A p: p = R^{-1} v, and the scale of the stored u: u_next = A p - (alpha / beta) u_stored
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) sh[j] = L.v[j];
  solve_r(L.R, L.ldr, n, sh);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    L.p[j] = sh[j];
    L.z[j] = 0.0;
  }
  if (threadIdx.x == 0) {
    sc[kLsqrC] = (beta > 0.0) ? -alpha / beta : 0.0;
    sc[kLsqrAlpha] = alpha;
    sc[kLsqrBeta2] = 0.0;
    if (alpha == 0.0 || beta == 0.0) sc[kLsqrDone] = 1.0;
    sc[kLsqrIters] += first ? 0.0 : 1.0;
  }
}

// x = x0 + R^{-1} y (FP64), one CTA.
__global__ void __launch_bounds__(512) lsqr_finish_kernel(const LsqrLaunch L) {
  __shared__ double sh[kLsqrMaxN];
  for (int64_t j = threadIdx.x; j < L.n; j += blockDim.x) sh[j] = L.y[j];
  solve_r(L.R, L.ldr, L.n, sh);
  for (int64_t j = threadIdx.x; j < L.n; j += blockDim.x) L.x[j] = L.x0[j] + sh[j];
}

// p = x0 (as the vector the residual kernel multiplies), from the FP32 sketch-and-solve solution.
__global__ void lsqr_start_kernel(const LsqrLaunch L, const float* x0f) {
  for (int64_t j = threadIdx.x; j < L.n; j += blockDim.x) {
    L.x0[j] = (double)x0f[j];
    L.p[j] = (double)x0f[j];
    L.z[j] = 0.0;
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < kLsqrScalars; ++q) L.sc[q] = 0.0;
}

int64_t av_grid(int64_t m, int sms) { return std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8)); }

// A^T u with the smallest per-lane column count that covers n.
void launch_atu(const LsqrLaunch& L, int sms, cudaStream_t st) {
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((L.m + 255) / 256, (int64_t)sms * 4));
  if (L.n <= 32) lsqr_atu_kernel<1><<<grid, 256, 0, st>>>(L);
  else if (L.n <= 64) lsqr_atu_kernel<2><<<grid, 256, 0, st>>>(L);
  else if (L.n <= 128) lsqr_atu_kernel<4><<<grid, 256, 0, st>>>(L);
  else if (L.n <= 256) lsqr_atu_kernel<8><<<grid, 256, 0, st>>>(L);
  else lsqr_atu_kernel<16><<<grid, 256, 0, st>>>(L);
}

}  // namespace

cudaError_t lsqr_start(const LsqrLaunch& L, const float* b, const float* x0f, int sms, cudaStream_t st,
                       int32_t* launches) {
  lsqr_start_kernel<<<1, 512, 0, st>>>(L, x0f);
  // u = b - A x0, ||u||^2
  lsqr_av_kernel<<<(unsigned)av_grid(L.m, sms), 256, 2 * L.n * sizeof(float), st>>>(L, b);
  launch_atu(L, sms, st);
  lsqr_step_kernel<<<1, 512, 0, st>>>(L, 1);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

cudaError_t lsqr_iterate(const LsqrLaunch& L, int sms, cudaStream_t st, int32_t* launches) {
  // u <- A p + c u with c = -alpha / beta, written by the previous step kernel
  lsqr_av_kernel<<<(unsigned)av_grid(L.m, sms), 256, 2 * L.n * sizeof(float), st>>>(L, nullptr);
  launch_atu(L, sms, st);
  lsqr_step_kernel<<<1, 512, 0, st>>>(L, 0);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

cudaError_t lsqr_finish(const LsqrLaunch& L, cudaStream_t st, int32_t* launches) {
  lsqr_finish_kernel<<<1, 512, 0, st>>>(L);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

}  // namespace sk
