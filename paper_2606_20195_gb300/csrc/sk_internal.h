// Internal launch interfaces shared by the translation units of libsk (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sk {

struct TileDesc;

struct TileLaunch {
  const void* A;    // elements of type a_type (0 FP32, 1 binary16, 2 bfloat16)
  int32_t a_type = 0;
  void* Y;
  int64_t lda, n, row_begin, row_end;  // global rows [row_begin, row_end); A row 0 = row_begin
  int64_t d;
  int32_t k, rule;
  uint64_t seed;
  float scale;
  int64_t R;        // chunk rows
  int32_t NC;       // columns per work item (4, 8, 16, 32)
  int32_t kb;       // blocks per block group
  int32_t threads;  // threads per CTA
  int32_t grid;     // CTAs (0 = automatic)
  int32_t slices;   // work items per chunk (> 1: two-level combine through P)
  float* P;         // chunk totals, launch_P_floats(L) FP32 (slices > 1 or glob); zero on entry and on exit
  unsigned* status;   // sticky device status word (may be null)
  int64_t col_off;    // global column index of column 0 (keys the rounding random bits)
  int32_t allow_tma;  // stage A through TMA when its layout allows it
  int32_t depth;      // TMA ring slots per warp (1..4)
  int32_t mb;         // hash rounds per TMA box (1, or more when every work item takes the fast path)
  int32_t lr = 0;     // 1: lane-row scatter (one block group; used only when A is staged through TMA)
  int32_t own = 0;    // 1: owner kernel (NC = 32, kb = 1 or 2 blocks per item, A through TMA)
  int32_t vec = 0;    // 1: n = 1 vector path of the tile kernel (NC = 4, no TMA)
  int32_t glob = 0;   // 1: global-accumulator kernel (chunk totals in P, any d); needs P
  int32_t reg = 0;    // 1: register kernel (FP32 A through TMA, 32 columns x 1024 output rows per item); needs P
  int32_t reg_nsub = 0, reg_cap = 0;  // register kernel: TMA copies per staged box, list entries per output row
  int32_t no_finish = 0;  // 1: leave the chunk totals in P (no chunk-finish launch); P is then the caller's
};

// Shared-memory bytes the tile kernel needs for (B, kb, NC, threads, k, ring depth, rounds per box).
size_t tile_smem_bytes(int64_t B, int32_t kb, int32_t NC, int32_t threads, int32_t k, int32_t depth, int32_t mb = 1);
// Encode a 2-D tensor map over A (n columns, `rows` rows, row stride lda, element type a_type) with box
// NC x RB; false if the layout does not allow TMA (A not 16-byte aligned, row stride or box width not
// a multiple of 16 bytes, too many rows).
bool encode_a_map(void* map, const void* A, int32_t a_type, int64_t lda, int64_t n, int64_t rows, int32_t NC,
                  int32_t RB);
int32_t tile_slots(int32_t NC, int32_t kb);
// Add the chunk totals of P (chunk-major, d x n FP32 each, chunks [t_first, t_first + chunks)) into
// Y in ascending chunk order with the rule's scaling and rounding, and clear P (one launch).
cudaError_t launch_chunk_finish(const TileDesc& D, int32_t rule, float* P, int64_t t_first, int64_t chunks,
                                cudaStream_t st, int32_t* launches);
// Enqueue the chunked tile kernel (atomic flush). Returns a CUDA error code.
cudaError_t launch_tile(const TileLaunch& L, cudaStream_t st, int32_t* launches);
// Owner kernel (sk_own.cu): shared-memory bytes for kb blocks of B rows, threads per CTA, resident
// CTAs per SM, and the launch (L.NC == 32, L.kb in {1, 2}; fails if A cannot go through TMA).
size_t own_smem_bytes(int64_t B, int32_t kb);
int32_t own_threads();
int32_t own_ctas_per_sm(int32_t rule, size_t smem);
cudaError_t launch_own(const TileLaunch& L, cudaStream_t st, int32_t* launches);
// Chunks, column groups and block groups of a launch.
void tile_geometry(const TileLaunch& L, int64_t* chunks, int32_t* ncg, int32_t* nbg);
// Passes of the global-accumulator kernel: column slabs of *ns columns and batches of *cb chunks,
// chosen so that the chunk totals of one pass (cb x d x ns FP32) stay resident in L2.
void global_passes(const TileLaunch& L, int64_t* ns, int64_t* cb);
// FP32 elements of chunk-total scratch P a launch needs (0: none).
int64_t launch_P_floats(const TileLaunch& L);
// The global-accumulator kernel and its chunk finish, in passes (sk_global.cu); needs L.P.
cudaError_t launch_global(const TileLaunch& L, cudaStream_t st, int32_t* launches);
// Register kernel (sk_reg.cu): shared-memory bytes for a box of nsub TMA copies, lists of cap entries
// and overflow lists of ovf_cap entries; threads per CTA; output rows per work item; blocks of S that
// reach the widest group of output rows; the box and capacity for a sketch of d rows and block height
// B within `smem_limit` bytes (cap_fixed > 0 imposes the capacity; false if nothing fits); and the
// launch (its chunk finish included; needs L.P).
size_t reg_smem_bytes(int32_t nsub, int32_t cap, int32_t ovf_cap);
int32_t reg_threads();
int32_t reg_targets();
int32_t reg_blocks_per_group(int64_t d, int64_t B);
bool reg_choose_box(int64_t d, int64_t B, size_t smem_limit, int32_t cap_fixed, int32_t* nsub, int32_t* cap);
cudaError_t launch_reg(const TileLaunch& L, cudaStream_t st, int32_t* launches);
// Resident CTAs per SM of the tile kernel for (rule, threads, dynamic shared memory).
int32_t tile_ctas_per_sm(int32_t rule, int32_t threads, size_t smem);

struct LiteralLaunch {
  const void* A;
  int32_t a_type = 0;
  void* Y;
  int64_t lda, n, row_begin, row_end, d;
  int32_t k, rule;
  uint64_t seed;
  float scale;
  int64_t col_off;
};
cudaError_t launch_literal(const LiteralLaunch& L, cudaStream_t st, int32_t* launches);

struct DetLaunch {
  const void* A;
  int32_t a_type = 0;
  void* Y;
  float* P;  // d x n FP32 scratch, zeroed by the launcher
  int64_t lda, n, row_begin, row_end, d;
  int32_t k, rule;
  uint64_t seed;
  float scale;
  int64_t R;
  int64_t col_off;
};
cudaError_t launch_det(const DetLaunch& L, cudaStream_t st, int32_t* launches);

cudaError_t launch_pattern(int64_t d, int32_t k, uint64_t seed, int64_t i0, int64_t cnt, int32_t* rows,
                           int8_t* signs, cudaStream_t st);

// FP64 sketch-and-solve back end: QR of [SA | Sb] (d x (n+1)), x = R^-1 (Q^T Sb)[:n].
struct SolveLaunch {
  const void* SA;   // d x n, row stride lda_sa; float, binary16 or bfloat16 (rule), or FP64 (src_fp64)
  const void* Sb;   // d values with stride sb_stride, same type
  int64_t lda_sa = 0, sb_stride = 1;
  int32_t rule;
  int32_t src_fp64 = 0;  // 1: SA and Sb are FP64 (a stack of [R | c] factors of a tree level)
  int32_t solve_x = 1;   // 1: back substitution into x and kappa; 0: write [R | c] only (zero below the diagonal)
  int64_t d, n;
  double* part;     // scratch: partial sums, (ncta) * (n + 2) doubles
  double* R;        // scratch: n x (n+1) doubles (R and Q^T Sb)
  double* bcast;    // scratch: n doubles
  unsigned* bar;    // scratch: solve_bar_bytes() of barrier counters, zeroed by the launcher
  unsigned* status; // sticky status word
  double* kappa;    // out: max|R_ii| / min|R_ii|
  float* x;         // out: n floats
  int32_t ncta;
  long long wait_cycles = 0;  // bound on each grid-barrier wait in SM clock cycles (0: about two seconds)
};
// CTAs and rows per CTA the QR kernel will use for (d, n); 0 CTAs if unsupported.
int32_t solve_ctas(int64_t d, int64_t n, int32_t sms, size_t smem_optin);
// Rows one QR launch can hold in shared memory for n columns (0 if n is unsupported).
int64_t solve_rows_cap(int64_t n, int32_t sms, size_t smem_optin);
// Bytes of the grid-barrier counters a QR launch uses.
size_t solve_bar_bytes();
cudaError_t launch_solve(const SolveLaunch& L, cudaStream_t st, int32_t* launches);

// Sketch-and-precondition LSQR (sk_lsqr.cu). Device scalars (FP64) of the recurrence:
constexpr int kLsqrMaxN = 512;
enum : int {
  kLsqrBeta2 = 0,   // ||u||^2 accumulated by the matvec
  kLsqrC = 1,       // -alpha / beta, the scale of the stored u in the next matvec
  kLsqrPhibar = 2,
  kLsqrRhobar = 3,
  kLsqrAlpha = 4,
  kLsqrAnorm2 = 5,  // estimate of ||A R^{-1}||_F^2
  kLsqrBnorm = 6,   // ||b - A x0||
  kLsqrRnorm = 7,   // estimate of ||b - A x||
  kLsqrArnorm = 8,  // estimate of ||(A R^{-1})^T (b - A x)||
  kLsqrIters = 9,
  kLsqrDone = 10,   // 1: alpha or beta vanished (exact solution reached)
  kLsqrScalars = 16
};
struct LsqrLaunch {
  const float* A;
  int64_t lda, m, n;
  const double* R;  // n x n upper triangular R of the sketch's QR, row stride ldr
  int64_t ldr;
  double* u;        // storage of m doubles: u as (hi, lo) float pairs, first m hi then m lo
  double *v, *w, *y, *p, *z, *x0;  // n each
  double* x;        // out: n
  double* sc;       // kLsqrScalars
};
// Start (x0 from the FP32 sketch-and-solve solution; r0 = b - A x0; first step), one iteration, and
// x = x0 + R^{-1} y.
cudaError_t lsqr_start(const LsqrLaunch& L, const float* b, const float* x0f, int sms, cudaStream_t st,
                       int32_t* launches);
cudaError_t lsqr_iterate(const LsqrLaunch& L, int sms, cudaStream_t st, int32_t* launches);
cudaError_t lsqr_finish(const LsqrLaunch& L, cudaStream_t st, int32_t* launches);

// Batched persistent kernel.
struct BatchDesc;     // device-side item descriptor (sk_batch.cu)
struct BatchWork;     // device-side work item
cudaError_t launch_batch(const void* descs, const void* work, int64_t nwork, int32_t* counter, const void* zero_list,
                         int32_t nzero, int32_t rule, int32_t threads, size_t smem, int32_t grid, int64_t acc_floats,
                         int32_t slot_bytes, int32_t depth, unsigned* status, cudaStream_t st, int32_t* launches);

}  // namespace sk
