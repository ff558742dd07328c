/*
 * sk.h — C ABI of the GB300 SparseStack sketching library (libsk.so).
 *
 * The library forms Y = S*A for a tall matrix A (m x n, m >> n; FP32, or binary16 / bfloat16 through
 * sk_apply_typed) with a SparseStack sparse oblivious subspace embedding S (d x m): every column of S
 * holds exactly k nonzeros of value +-1/sqrt(k), one in each block of B = d/k consecutive rows;
 * k = 1 is CountSketch (paper Sec. 2.2, Definition of SparseStack; Sec. 4.1 for the block ranges and
 * the scaling). The sum is accumulated in FP32, or stored in binary16 under deterministic
 * round-to-nearest, exact stochastic or dithered rounding, or in bfloat16 (paper Sec. 4.2). S is never
 * stored: the kernels regenerate it from a counter-based hash of (seed, row, block). On top of the
 * sketch: sketch-and-solve and sketch-and-precondition least squares (Sec. 5.1, 5.3) and batched
 * uneven sketches.
 *
 * Conventions for every entry point
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers. The caller owns
 *     every buffer it passes; the library never frees them. A plan owns only its own scratch.
 *   - A is row-major with row stride lda >= n elements (A[i*lda + c]); Y is row-major d x n with
 *     row stride n; b is a vector of m floats; x is a vector of n floats.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Device work is
 *     enqueued on it; calls return once the work is enqueued, except where stated.
 *   - Arguments are validated before any work is enqueued; an invalid call enqueues nothing and
 *     returns SK_ERR_INVALID_ARG (or SK_ERR_UNSUPPORTED for valid but unsupported sizes).
 *     sk_last_error() then holds a message for the calling thread. Asynchronous device faults
 *     surface as SK_ERR_CUDA on a later call. Nothing aborts the process.
 *   - A plan may be used from one host thread at a time; distinct plans are independent.
 */
#ifndef SK_H_
#define SK_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SK_API __attribute__((visibility("default")))
#else
#define SK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SK_OK = 0,
  SK_ERR_INVALID_ARG = 1, /* bad sizes, null or misaligned pointers, unknown keys */
  SK_ERR_UNSUPPORTED = 2, /* valid request outside what this build implements (limits below) */
  SK_ERR_OOM = 3,         /* device or host allocation failed */
  SK_ERR_CUDA = 4,        /* a CUDA runtime call failed (message in sk_last_error) */
  SK_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  SK_ERR_NUMERIC = 6      /* a non-finite or singular value where a finite one is required */
} sk_status;

/* Accumulation / storage rule of Y (paper Sec. 4.2). */
typedef enum {
  SK_FP32 = 0,       /* Y is float; contributions added in FP32 */
  SK_FP16_RN = 1,    /* Y is binary16; each contribution rounded to nearest even */
  SK_FP16_SR = 2,    /* Y is binary16; exact stochastic rounding of each contribution */
  SK_FP16_DITHER = 3, /* Y is binary16; uniform dither of ~1 binary16 ulp, then nearest even */
  SK_BF16_RN = 4      /* Y is bfloat16; each contribution rounded to nearest even, bfloat16 adds */
} sk_rule;

/* Plan parameters for sk_plan_set / sk_plan_get. */
typedef enum {
  /* R, the chunk length in rows (>= 1). Contributions of the rows of one chunk that reach the same
   * output are summed in FP32 before the chunk total is scaled, rounded (FP16 rules) and added into
   * Y; chunk t holds the rows floor(i/R) == t. R = 1 is the paper's per-element scheme. 0 (the
   * default) lets the library pick R from the tuning table for (m, n, d, k). */
  SK_PARAM_CHUNK_ROWS = 1,
  /* Execution order. SK_MODE_ATOMIC (default): chunk totals are added into Y in whatever order the
   * GPU finishes them, and rows inside a chunk in any order. SK_MODE_DETERMINISTIC: the canonical
   * order (rows ascending inside a chunk, chunks ascending), bit for bit; slow, for verification.
   * SK_MODE_SERIAL_TILE: the fast tile kernel run by one warp of one CTA, which also follows the
   * canonical order; for verifying the fast kernel's arithmetic (slow). */
  SK_PARAM_MODE = 2,
  /* Global index of the first row of A passed to sk_apply (for row-sharded matrices: S and the
   * chunk index depend on the global row). Default 0. */
  SK_PARAM_ROW_OFFSET = 3,
  /* Kernel choice: SK_KERNEL_AUTO (default), SK_KERNEL_TILE (on-chip chunk accumulation with
   * shared-memory atomics), SK_KERNEL_LITERAL (one global atomic per element and nonzero, the
   * paper's design; R must be 1), SK_KERNEL_OWNER (on-chip chunk accumulation in which every
   * accumulator row has one owning warp: no atomics; needs n >= 32, A 16-byte aligned with lda a
   * multiple of 4, and B*128 bytes of shared memory per block; SK_ERR_UNSUPPORTED otherwise).
   * Inside a work item the owner kernel adds rows in ascending order, so a chunk processed as one
   * work item has exactly the canonical FP32 chunk total. SK_KERNEL_GLOBAL (chunk totals
   * accumulated in device memory with FP32 reductions, one warp per row; any block height).
   * SK_KERNEL_REGISTER (chunk accumulation in registers: every thread owns one output row x 32
   * columns of a 1024-row group, rows of A are routed to their owners through per-row lists in shared
   * memory, no floating-point atomics on chip; needs FP32 A, 16-byte aligned with lda a multiple of 4, and
   * atomic mode; SK_ERR_UNSUPPORTED otherwise). AUTO takes the register kernel for FP32 A with
   * k >= 2, n >= 32 and B = d/k <= 512 (except n >= 256 with k = 2) when A's layout allows TMA
   * (and neither SK_PARAM_TILE_COLS nor SK_PARAM_THREADS is set); otherwise the tile kernel, or the global kernel when a block of S is
   * too tall for the tile kernel's shared-memory accumulator, when the tile kernel would need several
   * block groups or only 4-column items of a matrix with n >= 256, and for n >= 256 at k <= 2. */
  SK_PARAM_KERNEL = 4,
  /* Columns per work item of the tile kernel (4, 8, 16 or 32; 0 = automatic). */
  SK_PARAM_TILE_COLS = 5,
  /* Threads per CTA of the tile kernel (128..1024, multiple of 32; 0 = automatic). */
  SK_PARAM_THREADS = 6,
  /* Read-only: number of kernel launches the last sk_apply/sk_solve enqueued. */
  SK_PARAM_LAST_LAUNCHES = 7,
  /* Read-only: the chunk length R the last sk_apply used. */
  SK_PARAM_LAST_CHUNK_ROWS = 8,
  /* Read-only: sticky status bits the sketch kernels of this plan set on the device (bit 0: a
   * bounded wait gave up, the results of that call are invalid). Reading it synchronizes the device.
   * After sk_apply_noalloc it also includes that call's status word (see sk_apply_noalloc). */
  SK_PARAM_DEVICE_STATUS = 9,
  /* Read-only: the kernel the last sketch ran: SK_KERNEL_TILE (1), SK_KERNEL_LITERAL (2),
   * SK_KERNEL_OWNER (3), SK_KERNEL_GLOBAL (4), 5 for the deterministic-mode kernel, or
   * SK_KERNEL_REGISTER (6); 0 before the first sketch. */
  SK_PARAM_LAST_KERNEL = 10,
  /* Rows per group of sk_solve's tree QR (0, the default: as many rows as the GPU's shared memory
   * holds, so a sketch that fits is factored by one launch). Values below 2n are raised to 2n. */
  SK_PARAM_SOLVE_GROUP_ROWS = 11,
  /* Register kernel: list entries per output row and staged box of rows (0, the default: about
   * lambda + 1.5 sqrt(lambda) for lambda = box rows / B, the mean entries per row and box, e.g. 3 at
   * B = 512, where about 6 % of the entries overflow; 1..64 imposes it). Rows
   * beyond a full list are added into the chunk totals by FP32 vector reductions instead, with the
   * same result up to FP32 summation order; small values exercise that path. */
  SK_PARAM_LIST_CAP = 12,
  /* Upper bound, in bytes, on the device scratch this plan holds (0, the default: none). A call that
   * would grow the plan's scratch beyond it returns SK_ERR_OOM before enqueueing any work (Y is left
   * as it was); for services that admit work under a device-memory budget. */
  SK_PARAM_SCRATCH_LIMIT = 13,
  /* Upper bound, in SM clock cycles, on each grid-barrier wait of sk_solve's QR kernel (0, the
   * default: about two seconds). A barrier that gives up ends the kernel and sk_solve_status returns
   * SK_ERR_TIMEOUT; small values exist to exercise that path. */
  SK_PARAM_SOLVE_WAIT_CYCLES = 14,
  /* Read-only: bytes of device scratch the plan holds now. */
  SK_PARAM_SCRATCH_BYTES = 15,
  /* m, the rows of A the plan's calls process (set at sk_plan_create; may be changed between calls).
   * S is a function of (seed, global row, block), so a plan serves matrices of any height with the
   * same S restricted to their rows; the default chunk length follows m. Its scratch is kept and
   * grown as needed, so one plan can serve a stream of requests of varying m without allocating
   * once it has seen the largest. */
  SK_PARAM_ROWS = 16,
  /* Batch only (sk_batch_set): chunk length of every item from its own m alone, at most this many
   * chunks per matrix and at least 4096 rows (a multiple of 256), instead of the tuning that looks at
   * the whole batch. A request's chunking, hence its rounding, then does not depend on what else is
   * in the batch (0, the default: tuned over the batch; SK_PARAM_CHUNK_ROWS, if set, wins). */
  SK_PARAM_ITEM_CHUNKS = 17
} sk_param;

enum { SK_MODE_ATOMIC = 0, SK_MODE_DETERMINISTIC = 1, SK_MODE_SERIAL_TILE = 2 };
enum {
  SK_KERNEL_AUTO = 0,
  SK_KERNEL_TILE = 1,
  SK_KERNEL_LITERAL = 2,
  SK_KERNEL_OWNER = 3,
  SK_KERNEL_GLOBAL = 4,
  /* 5 is the deterministic-mode kernel's number in SK_PARAM_LAST_KERNEL; it cannot be requested. */
  SK_KERNEL_REGISTER = 6
};

typedef struct sk_plan_s* sk_plan;

/* Library version as major*10000 + minor*100 + patch. */
SK_API int32_t sk_version(void);

/* Message describing the last failed call on this host thread ("" if none). */
SK_API const char* sk_last_error(void);

/*
 * sk_plan_create — a sketch plan for S (d x m) with k nonzeros per column, rounding rule `rule`
 * and sketch seed `seed` (paper Sec. 2.2 Definition of SparseStack, Sec. 4.1).
 *   d    rows of S, d >= 1, d % k == 0 (the paper assumes divisibility; others are rejected)
 *   m    columns of S = rows of A (>= 1); m * ceil(k/2) must stay below 2^62
 *   k    nonzeros per column, 1 <= k <= 64 (k = 1: CountSketch)
 *   rule one of sk_rule
 *   seed 64-bit seed; S and the rounding random bits are pure functions of it
 *   out  receives the plan (set to NULL on failure)
 * Host only: enqueues no device work and allocates no device memory.
 */
SK_API sk_status sk_plan_create(int64_t d, int64_t m, int32_t k, int32_t rule, uint64_t seed, sk_plan* out);

/* Set / read a plan parameter (sk_param). Unknown keys or out-of-range values: SK_ERR_INVALID_ARG. */
SK_API sk_status sk_plan_set(sk_plan plan, int32_t key, int64_t value);
SK_API sk_status sk_plan_get(sk_plan plan, int32_t key, int64_t* value);

/*
 * sk_apply — Y_dev = S * A_dev (paper Sec. 4.1 scatter, Sec. 4.2 FP16 variants).
 *   A_dev  device, m x n FP32 rows with stride lda (>= n); 16-byte alignment of A_dev and
 *          lda % 4 == 0 enable vector loads (other layouts are accepted and run slower)
 *   n      columns, 1 <= n <= 65535
 *   Y_dev  device, d x n, float (SK_FP32) or binary16 (FP16 rules), 4-byte aligned. Overwritten:
 *          the call zeroes Y on `stream` before accumulating.
 * The rows processed are the plan's m rows starting at global row SK_PARAM_ROW_OFFSET.
 */
SK_API sk_status sk_apply(sk_plan plan, const float* A_dev, int64_t lda, int64_t n, void* Y_dev, void* stream);

/* Element types of A for sk_apply_typed. */
enum { SK_A_FP32 = 0, SK_A_FP16 = 1, SK_A_BF16 = 2 };

/*
 * sk_apply_typed — Y_dev = S * A_dev for A stored as FP32, binary16 or bfloat16 (a_type one of
 * SK_A_FP32, SK_A_FP16, SK_A_BF16). 16-bit inputs move half the bytes of A; every value is converted
 * exactly to FP32 as it is loaded, so the result is that of sk_apply on the FP32 copy of A (bit for
 * bit in SK_MODE_DETERMINISTIC and SK_MODE_SERIAL_TILE). The paper's scheme reads FP32 A and names
 * lower-precision formats only for the accumulation (Sec. 4.2); this entry point extends the input.
 *   A_dev  device, m x n elements of a_type with row stride lda (>= n), aligned to the element
 *          size; TMA staging needs a 16-byte-aligned A_dev and lda * element size a multiple of 16
 *          (other layouts are accepted and run slower)
 *   n, Y_dev, stream: as for sk_apply.
 * Errors: SK_ERR_INVALID_ARG for an unknown a_type or a misaligned A_dev; SK_ERR_UNSUPPORTED with
 * SK_KERNEL_OWNER and a 16-bit A (the owner kernel reads FP32 only).
 */
SK_API sk_status sk_apply_typed(sk_plan plan, const void* A_dev, int32_t a_type, int64_t lda, int64_t n, void* Y_dev,
                                void* stream);

/*
 * sk_apply_host — the same result from HOST buffers: A_host is copied to the device in row tiles
 * (pinned memory gives overlapped asynchronous copies; pageable memory is accepted), the tiles are
 * sketched as they arrive, and Y is copied back to Y_host. Blocks until Y_host is written.
 * Device staging buffers are allocated on first use and kept by the plan.
 */
SK_API sk_status sk_apply_host(sk_plan plan, const float* A_host, int64_t lda, int64_t n, void* Y_host, void* stream);

/*
 * sk_solve — sketch-and-solve least squares (paper Sec. 5.1): x = argmin ||(S A) x - (S b)||_2.
 * SA and Sb are formed with this plan's S and rule (Sb uses the same chunking, as column n of
 * [A | b]), converted to FP64, factored by a Householder QR on the device, and x is recovered by
 * Q^T (S b) and back substitution, all in FP64; x is written as FP32. A sketch taller than the
 * GPU's shared memory holds is factored as a tree: groups of rows are factored separately and
 * their triangular factors (with Q^T Sb) stacked and factored again (SK_PARAM_SOLVE_GROUP_ROWS).
 *   A_dev, lda, n as in sk_apply; requires n <= d and n <= 1024.
 *   b_dev  device, m floats; x_dev device, n floats.
 * Device scratch (d x (n+1) sketch and FP64 workspace) is allocated on first use and grown as
 * needed; calls after the first with the same or smaller n allocate nothing.
 * A rank-deficient SA (a zero pivot in the QR) is reported by sk_solve_status.
 */
SK_API sk_status sk_solve(sk_plan plan, const float* A_dev, int64_t lda, int64_t n, const float* b_dev, float* x_dev,
                   void* stream);

/*
 * sk_solve_sketched — the FP64 back end of sk_solve on a sketch the caller already holds (paper
 * Sec. 5.1: QR of S A, then x from R x = (Q^T S b)[:n]). For services that form the sketches of many
 * requests in one batched launch (sk_batch_launch over [A_i | b_i]) and then solve each.
 *   SAb_dev: device, d x (n+1) values of the plan's output type (FP32 for SK_FP32, binary16 or
 *     bfloat16 otherwise), row-major with row stride ld >= n + 1 elements: columns 0..n-1 are S A,
 *     column n is S b. Read only. d is the plan's d; requires n <= d and n <= 1024.
 *   x_dev: device, n floats (output).
 * Uses and grows the plan's FP64 workspace as sk_solve does (no allocation once it has seen this n);
 * the plan's m, k and seed play no part. Status and kappa: sk_solve_status. Errors: as sk_solve,
 * synchronously for arguments; nothing is enqueued on an error.
 */
SK_API sk_status sk_solve_sketched(sk_plan plan, const void* SAb_dev, int64_t ld, int64_t n, float* x_dev,
                                   void* stream);

/* Status of the last sk_solve or sk_solve_sketched on this plan: synchronizes `stream`, then reads the device status
 * word. SK_ERR_NUMERIC: SA was rank deficient (zero pivot; x was set to NaN). SK_ERR_TIMEOUT: a
 * grid barrier of the QR kernel gave up waiting. Also writes the FP64 estimate
 * kappa(SA) ~ max|R_ii| / min|R_ii| (>= 1) if kappa != NULL. */
SK_API sk_status sk_solve_status(sk_plan plan, double* kappa, void* stream);

/*
 * sk_solve_precond — sketch-and-precondition least squares: x = argmin ||A x - b||_2 in FP64.
 * The sketch S [A | b] and its FP64 QR are formed exactly as by sk_solve (same plan, rule and
 * chunking); R then serves as a right preconditioner for LSQR (Paige and Saunders, 1982) on A itself,
 * started from the sketch-and-solve solution. The paper's discussion names this use of the sketch
 * (R of S A as a preconditioner) beside sketch-and-solve (Sec. 5.1). Since A R^{-1} has singular
 * values within the sketch's distortion of 1, a few tens of iterations reach the least-squares
 * solution of A, whatever the rounding rule of the sketch.
 *   A_dev, lda, n, b_dev: as for sk_solve (n <= 512). x_dev: n doubles on the device (output).
 *   max_iters: iteration limit (<= 0: 100). tol: stop when the estimate of
 *     ||(A R^{-1})^T r|| / (||A R^{-1}||_F ||r||) <= tol or ||r|| <= tol ||b - A x0|| (<= 0: 1e-10).
 *   iters_out (may be NULL): iterations used.
 * Every iteration runs on the GPU in FP64; the call synchronizes `stream` every few iterations to
 * test convergence and returns when x_dev is written. Scratch (m + 9n doubles) is plan-owned.
 * Errors: as sk_solve; SK_ERR_NUMERIC if S A is rank deficient (no preconditioner).
 */
SK_API sk_status sk_solve_precond(sk_plan plan, const float* A_dev, int64_t lda, int64_t n, const float* b_dev,
                                  double* x_dev, int32_t max_iters, double tol, int32_t* iters_out, void* stream);

/*
 * sk_materialize_S — write the nonzero pattern of S for rows [i0, i0+cnt) on the device:
 * rows_dev[(i-i0)*k + j] = target row of block j (int32), signs_dev[...] = +1 or -1 (int8).
 * The same generator the sketch kernels use; for verification of the pattern.
 */
SK_API sk_status sk_materialize_S(sk_plan plan, int64_t i0, int64_t cnt, int32_t* rows_dev, int8_t* signs_dev,
                           void* stream);

/*
 * Batched uneven sketches in one persistent launch (row tiles of every matrix drawn from one
 * device work list). item i sketches A_i (m_i x n_i, stride lda_i) into Y_i (d_i x n_i) with
 * k_i nonzeros per column, seed_i, and the batch's common rule. Items are independent.
 * The work list is built on the host and copied to the device inside the call; a batch object
 * keeps it so the launch can be replayed (and captured in a CUDA graph) with sk_batch_launch.
 */
typedef struct {
  const float* A_dev;
  void* Y_dev;
  int64_t m, n, lda, d;
  int32_t k;
  int32_t pad_;
  uint64_t seed;
} sk_batch_item;

typedef struct sk_batch_s* sk_batch;

/* Build a batch: validates every item, chooses tiles (threads, columns per work item, chunk rows)
 * from the tuning table unless overridden by sk_batch_set, and uploads the work list.
 * Allocates device memory for the work list (kept by the batch). */
SK_API sk_status sk_batch_create(const sk_batch_item* items, int32_t count, int32_t rule, sk_batch* out);
/* Replace the items of a batch (same rule and overrides). The next sk_batch_launch rebuilds the
 * work list and uploads it on its stream, reusing the batch's device buffers when they are large
 * enough (they grow otherwise), so a service that sketches a new set of requests at every
 * scheduling step keeps one batch object per rule instead of creating and destroying one per step
 * (sk_batch_destroy synchronizes the device). The previous launch of this batch must have
 * completed (its work list is overwritten in place). */
SK_API sk_status sk_batch_rebind(sk_batch batch, const sk_batch_item* items, int32_t count);
/* Override the tile choice: key is SK_PARAM_TILE_COLS, SK_PARAM_THREADS, SK_PARAM_CHUNK_ROWS or
 * SK_PARAM_ITEM_CHUNKS; must be called before the first sk_batch_launch after a create or a rebind. */
SK_API sk_status sk_batch_set(sk_batch batch, int32_t key, int64_t value);
/* Zero every Y_i and run the persistent kernel on `stream`. The first launch after sk_batch_create
 * or sk_batch_rebind builds the work list and uploads it on `stream` (allocating or growing the
 * batch's device buffers if needed); later launches allocate nothing and never synchronize, so such
 * a launch can be captured into a CUDA graph and replayed. */
SK_API sk_status sk_batch_launch(sk_batch batch, void* stream);
/* Work-list statistics: number of work items and total bytes of A the batch reads. */
SK_API sk_status sk_batch_info(sk_batch batch, int64_t* work_items, int64_t* bytes_A);
SK_API void sk_batch_destroy(sk_batch batch);

/*
 * sk_apply_noalloc — the same result as sk_apply in SK_MODE_ATOMIC (same kernel, same chunking),
 * for callers that must not allocate device memory: code running where cudaMalloc is forbidden or
 * unsafe (inside an allocator or memory-pool callback, a real-time or fixed-footprint service whose
 * memory is budgeted up front, an embedding application that owns all device memory). The paper has
 * no counterpart; this is an interface variant of the sketch call.
 *
 * Instead of plan-owned scratch, the kernels' scratch (per-chunk FP32 totals and the status word)
 * lives in one fixed static device array of 16 MiB in this library. The caller still passes A and Y
 * exactly as for sk_apply. The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine; it only enqueues memsets and the kernels on `stream` (the same launches as sk_apply).
 *   - Every call looks up the device address of that array (cudaGetSymbolAddress) with the
 *     calling thread's current device; the first lookup on a device may load the library's device
 *     code there, so make the first call on each device before any stream capture on it.
 *   - The kernels' status word lives in the array too: after a call, SK_PARAM_DEVICE_STATUS of the
 *     plan (which synchronizes the device) reports the status of the most recent no-allocation call
 *     on the current device (bit 0: a bounded wait gave up and that call's Y is invalid). The word is
 *     cleared at the start of every call.
 *   - Sizes whose scratch exceeds 16 MiB (chunks x d x n x 4 bytes when chunks are split across CTAs,
 *     the chunk totals of one pass for the global kernel) are rejected with SK_ERR_UNSUPPORTED and a
 *     message; use sk_apply for those.
 *   - Every call on a device shares the one array: calls that overlap on the GPU (different streams,
 *     or different host threads) race and give wrong results. Serialize them on one stream.
 *   - Only SK_MODE_ATOMIC is supported, with the kernel AUTO picks or the tile, owner or global kernel
 *     (SK_ERR_UNSUPPORTED for the deterministic modes and the literal kernel).
 */
SK_API sk_status sk_apply_noalloc(sk_plan plan, const float* A_dev, int64_t lda, int64_t n, void* Y_dev, void* stream);

/*
 * Row-sharded sketches (the one exchange step of a multi-GPU sketch). S depends only on the global row
 * index, so Y = sum over shards of S[:, rows_g] A[rows_g, :]; summing must happen before the rounding
 * of the 16-bit rules, on the FP32 chunk totals (the paper's Sec. 4.1 scatter, with the chunked
 * pre-combine; Sec. 4.2 rounding after the sum). A shard's plan covers its rows: m rows starting at
 * global row SK_PARAM_ROW_OFFSET, and SK_PARAM_CHUNK_ROWS (R) must be set to the same value on every
 * shard. P is a device buffer of nchunks x d x n FP32 values, chunk-major (d x n each, row stride n),
 * 16-byte aligned; slot q holds global chunk t0 + q (the rows [t R, (t+1) R) of chunk t).
 *
 * sk_apply_partials — adds into P_dev the FP32 chunk totals of the plan's rows (it does not clear P;
 *   start from zero). Nothing is rounded. The plan's chunks must lie in [t0, t0 + nchunks).
 *   Atomic mode only (SK_ERR_UNSUPPORTED otherwise); A_dev, lda, n as for sk_apply.
 * sk_finish_partials — Y_dev = the sketch from the summed chunk totals: for every output, the chunk
 *   totals of P_dev in ascending chunk order, each scaled by fl32(1/sqrt(k)), rounded by the plan's rule
 *   and added into Y (zeroed first), exactly as sk_apply finishes its own chunk totals. Clears P_dev.
 * With one shard the pair gives sk_apply's result (same chunk totals up to the FP32 summation order
 * inside a chunk); with several, sum the shards' P (an all-reduce in FP32) between the two calls.
 */
SK_API sk_status sk_apply_partials(sk_plan plan, const float* A_dev, int64_t lda, int64_t n, float* P_dev, int64_t t0,
                                   int64_t nchunks, void* stream);
SK_API sk_status sk_finish_partials(sk_plan plan, float* P_dev, int64_t t0, int64_t nchunks, int64_t n, void* Y_dev,
                                    void* stream);

/* Release the plan and its device scratch (synchronizes the device first). NULL is a no-op. */
SK_API void sk_destroy(sk_plan plan);

#ifdef __cplusplus
}
#endif

#endif /* SK_H_ */
