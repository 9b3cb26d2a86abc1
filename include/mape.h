/*
 * mape.h -- C ABI of the GB300 implementation of MAPE's data-parallel hot
 * path (Multi-start Augmentation via Parallel Extraction, Liu, Wang & Yang,
 * "Parallel Graver Basis Extraction for Nonlinear Integer Optimization").
 *
 * Problem (Eq. (1), §1):  min f(x)  s.t.  A x = b,  l <= x <= u,  x in Z^n,
 * with f(x) = x^T Q x + c^T x + sum_i w_i x_i^4 (Q symmetric, integer; w >= 0
 * optional).  B (n x d, d = n - m) is a basis of the integer kernel
 * Ker_Z(A) = L(B) (Theorem 3.2, §3.1).
 *
 * Two layers:
 *   1. Stage entry points (mape_project_starts ... mape_augment_run).  All
 *      array arguments are DEVICE pointers owned by the caller; sizes are host
 *      integers.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *      default stream).  Entry points that return a count through a host
 *      pointer synchronise the stream before returning; the others are
 *      asynchronous.  Scratch memory is passed in as (workspace, bytes) and its
 *      size is given by the matching *_workspace_bytes query.
 *   2. The instance handle (mape_create_instance ... mape_destroy).  All array
 *      arguments are HOST pointers owned by the caller and copied during the
 *      call; the library owns every device buffer of the handle, allocated
 *      through the allocator set with mape_set_allocator (default:
 *      stream-ordered allocation on the handle's stream from a library pool
 *      that keeps freed memory).  extract_directions and
 *      augment return at once and run on a worker thread of the handle;
 *      mape_poll reads progress, mape_wait blocks with a timeout.
 *
 * Every call returns MAPE_OK (0), a negative error code, or a positive
 * warning code.  Layouts are row-major (C order) unless stated.
 * Direction sets are stored as int8 rows of pitch `ldg` bytes (ldg a multiple
 * of 16, ldg >= n), which requires max_i (u_i - l_i) <= 127: with condition C4
 * (l - u <= g <= u - l, §3) every collected direction then fits in int8.
 */
#ifndef MAPE_H_
#define MAPE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define MAPE_OK                    0
#define MAPE_ERR_INVALID_ARG      -1  /* NULL pointer, negative size, bad enum */
#define MAPE_ERR_SHAPE            -2  /* sizes outside what the path supports */
#define MAPE_ERR_NOT_KERNEL_BASIS -3  /* A B != 0 (Theorem 3.2 precondition) */
#define MAPE_ERR_BOUNDS           -4  /* some u_i < l_i, or u - l > 127 */
#define MAPE_ERR_INFEASIBLE       -5  /* an augmentation start is not in S */
#define MAPE_ERR_OVERFLOW         -6  /* exact integer range of a stage exceeded */
#define MAPE_ERR_CAPACITY         -7  /* an output buffer or table is full */
#define MAPE_ERR_CUDA             -8  /* a CUDA runtime call failed */
#define MAPE_ERR_TIMEOUT          -9  /* mape_wait timed out / bounded wait gave up */
#define MAPE_ERR_STATE           -10  /* call not valid in the handle's phase */
#define MAPE_ERR_OOM             -11  /* device allocation failed */
#define MAPE_ERR_KERNEL_TEST     -12  /* a collected direction failed A g = 0 (C1) */
#define MAPE_ERR_NUMERIC         -13  /* an iterate left the exactly-rounded range */
#define MAPE_ERR_CANCELLED       -14  /* mape_cancel was called */

/* ---- precision of the extraction contractions ---------------------------- */
#define MAPE_PREC_FP32 0  /* comparator only, not a product path: the plain
                             FP32 single-instance baseline that the tensor-core
                             paths are measured against.  Per step, strict-FP32
                             cuBLAS GEMMs for B z, B^T sign(Bz), B round(z)
                             and unfused elementwise kernels, as a direct
                             PyTorch version of the method would run them    */
#define MAPE_PREC_BF16 1  /* tcgen05 BF16 MMAs with FP32 accumulation in TMEM,
                             persistent fused kernel over all T steps; z enters
                             the forward product as hi + lo (two BF16 terms),
                             accurate to about FP32                             */
#define MAPE_PREC_BF16X1 2 /* as MAPE_PREC_BF16 with z as one BF16 term (hi):
                             half the forward MMAs, 8-bit z in B z            */
#define MAPE_PREC_FP8 4    /* the streamed tensor-core kernels with the forward
                             product B z in FP8: z as e4m3 scaled per start
                             by a power of two (max |z| of each start lands in
                             [128, 256)), B as e4m3 (entries must be exact
                             in e4m3, e.g. |B_ij| <= 16; flag 8 otherwise),
                             kind::f8f6f4 MMAs with FP32 accumulation, 2 per
                             64 coordinates instead of 8 for MAPE_PREC_BF16;
                             z carries 4 significant bits in B z (sign(Bz)
                             is coarse), B round(z) stays exact in BF16 and
                             the gradient runs as for MAPE_PREC_BF16       */
#define MAPE_PREC_SPARSE 3 /* FP32 on CUDA cores for an identity-topped B =
                             [I ; B'] with sparse B' (compressed rows and
                             columns): one block per start with its z, m, v
                             in shared memory for all T steps             */
/* The BF16 precisions run one of two tensor-core implementations, with the
 * same arithmetic per step:
 *   resident: one persistent fused kernel for all T steps, B and the tile's
 *             z, m, v on chip; for tiles that fit (rows of B through the MMA
 *             and d at most 256, the operands within shared memory);
 *   streamed: three kernels per step (forward + map, collect, gradient +
 *             Adam) over tiles of 128 starts, with B and the state streamed
 *             through shared memory by bulk copies; any n, d <= 4096.
 * The resident kernel is chosen when it fits; OR-ing MAPE_PREC_STREAMED into
 * the precision forces the streamed one. */
#define MAPE_PREC_STREAMED 0x100
/* OR-ing MAPE_PREC_AUTOTUNE into a BF16 precision lets the library choose the
 * implementation and the streamed kernels' N-block widths (64, 128 or 256
 * rows of B per forward CTA, coordinates per gradient CTA) for this shape
 * (into MAPE_PREC_FP8: the widths of its streamed kernels only): the
 * first call for a (n, d, P rounded up to a power of two, precision) times a
 * few steps of every candidate on scratch copies of the call's state (inside
 * the workspace, which is larger with this bit) and keeps the fastest for the
 * process; later calls reuse it.  Results are those of the chosen
 * implementation; mape_autotune_lookup reports the choice and the probes. */
#define MAPE_PREC_AUTOTUNE 0x200
/* OR-ing MAPE_PREC_SPARSE_FWD into MAPE_PREC_BF16 runs the forward product
 * of the streamed path on the CUDA cores over the compressed rows of Bm, for
 * an identity-topped B = [I; Bm] whose Bm has density at most 1/16
 * (nnz(Bm) <= R d / 16; SHAPE otherwise): y = Bm z in FP32 from the full FP32
 * z (at least as accurate as the two BF16 terms); the gradient stays on the
 * tensor cores.  Implies MAPE_PREC_STREAMED. */
#define MAPE_PREC_SPARSE_FWD 0x400
#define MAPE_PREC_MASK 0xff

/* ---- hyper-parameters (§3.2, §4: lambda1 = 0.85, lambda2 = 1, lr = 0.003) - */
typedef struct {
  float lambda1, lambda2;      /* weights in Eq. (3)                            */
  float lr, eps;               /* Adam (Kingma & Ba) step size and epsilon      */
  double beta1, beta2;         /* Adam decay rates; double so that 1 - beta is
                                  formed exactly (0.999 is not an FP32 value:
                                  1 - 0.999f is off by 1.3e-5 relative)        */
  int32_t T;                   /* Adam steps per start                          */
  int32_t period;              /* collect every `period` steps (Algorithm 2)    */
  int32_t precision;           /* MAPE_PREC_*                                   */
  int32_t reserved;
  int64_t cand_capacity;       /* candidate-buffer rows of a handle (0:
                                  P * (T / period + 1), at most 2^23 rows and
                                  2 GiB per buffer)                          */
  int64_t max_aug_iters;       /* cap on Algorithm 1 iterations per call        */
} mape_config;

/* Fills `cfg` with the paper's values: lambda1 0.85, lambda2 1, lr 0.003,
 * beta1 0.9, beta2 0.999, eps 1e-8, T 1000, period 1, BF16. */
void mape_default_config(mape_config* cfg);

/* ========================================================================== *
 * Stage entry points (device pointers)                                        *
 * ========================================================================== */

/* a2 -- starting points (§3.2, Algorithm 2): z0 = (B^T B)^{-1} B^T g for every
 * sample row g of G0.
 *   B   [n x d] int32      kernel basis, full column rank
 *   G0  [P x n] float32    samples g ~ Uniform(l - u, u - l), one per start
 *   Z0  [P x d] float32    output starting points
 * Forms B^T B, factors it by Cholesky in FP32 on the device and solves.
 * Errors: INVALID_ARG, SHAPE (d > 4096), NUMERIC (B^T B not positive
 * definite in FP32), CAPACITY (workspace too small), CUDA.  Synchronous. */
size_t mape_project_workspace_bytes(int32_t n, int32_t d);
int mape_project_starts(const int32_t* B, int32_t n, int32_t d,
                        const float* G0, int32_t P, float* Z0,
                        void* workspace, size_t workspace_bytes, void* stream);

/* The two halves of mape_project_starts, for callers that project many
 * batches with the same B:
 *   prepare: W = B (B^T B)^{-1}  (W [n x d] float32, per instance; Cholesky
 *            in FP32; NUMERIC if B^T B is not positive definite).  Synchronous.
 *   apply:   Z0 = G0 W, i.e. z0 = W^T g per start (a tiled FP32 GEMM).
 *            Asynchronous. */
size_t mape_project_prepare_workspace_bytes(int32_t n, int32_t d);
int mape_project_prepare(const int32_t* B, int32_t n, int32_t d, float* W,
                         void* workspace, size_t workspace_bytes, void* stream);
int mape_project_apply(const float* W, int32_t n, int32_t d, const float* G0,
                       int32_t P, float* Z0, void* stream);

/* a3-a5 -- Eq. (3) and its gradient in FP32 for every start row z of Z:
 *   phi[p]      = ||B z||_1 + lambda1 sum_i (z_i - floor z_i)(ceil z_i - z_i)
 *                 + lambda2 max{1/||z||_inf - 1, 0}
 *   grad[p, :]  = B^T sign(B z) + lambda1 (ceil z + floor z - 2 z)
 *                 - lambda2 [||z||_inf < 1] sign(z_k) / ||z||_inf^2 e_k,
 *                 k the first index of max |z_j|; sign(0) = 0; zero at z = 0.
 *   B [n x d] int32, Z [P x d] float32, phi [P] float32 (+inf at z = 0),
 *   grad [P x d] float32.  Asynchronous. */
int mape_phi_grad(const int32_t* B, int32_t n, int32_t d, const float* Z,
                  int32_t P, float lambda1, float lambda2, float* phi,
                  float* grad, void* stream);

/* a3-a8 -- Algorithm 2 (§3.2), the parallel extraction loop, for T steps:
 * every start takes Adam steps on Eq. (3); after each step whose number is a
 * multiple of `period` the rounded point g = B round(z) (ties to even) is
 * tested for g != 0 and C4 (|g_i| <= span_i) and, if it passes and the
 * rounded point changed since that start's previous collection in this call
 * (the first collection of a call always counts), appended to `cand` in
 * canonical sign (first nonzero entry positive).  Repeated directions are
 * removed later by mape_dedup; skipping an unchanged rounding only avoids a
 * duplicate.
 * Continuing a run: pass the Z/M/V of the previous call and t0 = the number
 * of steps already taken (Adam bias correction uses t0 + 1 ... t0 + T).
 */
typedef struct {
  int32_t n, d, P;
  const int32_t* B;        /* [n x d] int32                                  */
  const int32_t* span;     /* [n] int32, u - l (C4), each in [0, 127]: device  */
                           /* memory, not checked by this call (a larger span  */
                           /* lets values beyond int8 into the candidate rows) */
  float* Z;                /* [P x d] in/out                                  */
  float* M;                /* [P x d] in/out, Adam first moment               */
  float* V;                /* [P x d] in/out, Adam second moment              */
  int32_t t0, T, period, precision;
  float lambda1, lambda2, lr, eps;
  double beta1, beta2;
  int8_t* cand;           /* [cand_cap x ldc] output rows                    */
  int32_t ldc;             /* row pitch in bytes, multiple of 16, >= n        */
  int32_t pad0;
  int64_t cand_cap;
  unsigned long long* cand_count; /* device counter, appended to (not reset)  */
  int32_t* flags;          /* device word, OR-ed: 1 = cand overflow (rows
                              beyond cand_cap are counted, not stored),
                              2 = |round(z)| > 256 met on the BF16 path (the
                              exactness bound of B round(z) in BF16; that
                              start's rounding is not collected),
                              4 = on the FP32 path, |round(z)| above
                              (2^24 - 1) / max_i sum_j |B_ij|, beyond which
                              B round(z) is not exact in FP32 (that start's
                              rounding is not collected)                 */
  float* dbg_phi;          /* optional [P]: Phi at the input point            */
  float* dbg_grad;         /* optional [P x d]: gradient at the input point   */
  void* workspace;
  size_t workspace_bytes;
} mape_extract_args;
/* Errors: INVALID_ARG, SHAPE (n or d above 4096 on the BF16 paths; n above
 * 49152 on the FP32 path; on the sparse path a B without identity top or a
 * start's state beyond shared memory), NUMERIC (sparse path: an entry of B'
 * beyond 2^23), CAPACITY (workspace), CUDA.  Asynchronous, except that the
 * BF16 and sparse paths synchronise `stream` once to inspect B (identity
 * top, exactness, sparsity) before the steps are queued. */
size_t mape_extract_workspace_bytes(int32_t n, int32_t d, int32_t P, int32_t precision);
int mape_extract(const mape_extract_args* args, void* stream);

/* a3-a8 for many instances at once (uneven n, d and P): every call of
 * `items` as in mape_extract (each with its own B, state, candidate buffer,
 * counter, flags and workspace of mape_extract_workspace_bytes), all with the
 * same t0, T, period and BF16 precision.  The calls that fit the resident
 * kernel run as one persistent launch per kernel variant (identity-topped or
 * general B, state in TMEM or not) over all their tiles; the others run the
 * streamed kernels with three launches per step covering all of them; all of
 * it is captured into one CUDA graph and launched (not on the legacy default
 * stream, which is not capturable: there the kernels are launched directly).
 * Each call's results are identical to its own mape_extract.  `workspace`
 * holds the batch's tables (mape_extract_batch_workspace_bytes).
 * Errors: as mape_extract, plus INVALID_ARG for differing t0, T, period or
 * precision, or an FP32 precision.  Synchronous. */
size_t mape_extract_batch_workspace_bytes(const mape_extract_args* items, int32_t count);
int mape_extract_batch(const mape_extract_args* items, int32_t count,
                       void* workspace, size_t workspace_bytes, void* stream);

typedef struct {
  int32_t path;             /* chosen: 0 resident fused kernel, 1 streamed,
                               2 streamed with the sparse CUDA-core forward   */
  int32_t wF, wG;           /* streamed: forward / gradient N-block widths    */
  int32_t candidates;       /* candidates that ran                            */
  int32_t probe_steps;      /* Adam steps each candidate was timed on         */
  int32_t cand_path[16], cand_wF[16], cand_wG[16];
  float probe_ms[16];       /* their times                                    */
} mape_tune_info;
/* The autotuned choice for a shape, or STATE if none was made yet. */
int mape_autotune_lookup(int32_t n, int32_t d, int32_t P, int32_t precision, mape_tune_info* out);
/* Forgets every autotuned choice of the process (extraction paths and the
 * lane counts of the augmentation scoring pass). */
void mape_autotune_clear(void);

/* a10 -- set union of Algorithm 2: removes repeated rows of `cand` (count
 * rows, pitch ldc, n meaningful bytes) with a device hash table, and writes
 * the distinct rows to `uniq` sorted lexicographically (signed bytes, first
 * entry most significant).  *K_out = number of distinct rows.
 * Errors: INVALID_ARG, CAPACITY (uniq_cap < distinct rows; *K_out is still
 * set to the needed count), CUDA.  Synchronous. */
size_t mape_dedup_workspace_bytes(int64_t count, int32_t ldc);
int mape_dedup(const int8_t* cand, int64_t count, int32_t n, int32_t ldc,
               int8_t* uniq, int64_t uniq_cap, int64_t* K_out,
               void* workspace, size_t workspace_bytes, void* stream);

/* mape_dedup without any device allocation (this entry point has no
 * counterpart in the paper; it is an interface for callers).  Some callers
 * cannot allocate device memory where they dedup: hosts that reserve all
 * device memory up front and forbid later allocations (a fixed memory budget
 * for a long-running loop), or plugins whose host owns the device allocator
 * and gives them none.  This variant takes no workspace: its scratch is a
 * static device array of 10 MiB inside the library, which every GPU that
 * loads the library holds until the process exits.
 *   Limit: count <= mape_dedup_static_max_rows() (2^18 rows, any ldc up to
 *   the stage's own limits); larger counts return MAPE_ERR_CAPACITY before
 *   any device work.
 *   The call is synchronous like mape_dedup: it reads the distinct count back
 *   to the host and synchronises `stream`.  It therefore cannot be made while
 *   a stream is being captured into a CUDA graph.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and caches it; a call
 *   that fails with a CUDA error forgets the cached address, and so must the
 *   caller's first call after a cudaDeviceReset (which invalidates it): such
 *   a call looks it up again.  Devices numbered 64 and above are refused with
 *   MAPE_ERR_INVALID_ARG.
 *   All calls share the array and it keeps the previous call's contents; the
 *   call clears what must start empty itself.  Calls that overlap on the GPU
 *   (different streams or threads at the same time) race on the array and
 *   must not be issued.
 * Arguments, output and errors otherwise as mape_dedup. */
int64_t mape_dedup_static_max_rows(void);
int mape_dedup_static(const int8_t* cand, int64_t count, int32_t n, int32_t ldc,
                      int8_t* uniq, int64_t uniq_cap, int64_t* K_out,
                      void* stream);

/* a10 for many candidate sets at once (the sets of a batch of instances):
 * item i is one mape_dedup call -- its own rows, count, n, ldc, output and
 * workspace of mape_dedup_workspace_bytes(count, ldc) -- and gets the same
 * output and K.  Every kernel of the stage runs once over the rows of all
 * sets (hash, insert, compaction, keys, the bitonic stages, the run sorts,
 * the gather), each thread, warp or block finding its set by binary search
 * over the launch's prefix table; `workspace` holds the batch's tables
 * (mape_dedup_batch_workspace_bytes(count)).  Per item: K (distinct rows)
 * and status (MAPE_OK, or CAPACITY when they exceed uniq_cap: nothing is
 * then written for that item, as in mape_dedup).  Returns the first item's
 * error, else INVALID_ARG / SHAPE for bad arguments (checked before any
 * device work) or CUDA.  Synchronous. */
typedef struct {
  const int8_t* cand;       /* [count x ldc] device                          */
  int64_t count;
  int32_t n, ldc;
  int8_t* uniq;             /* [uniq_cap x ldc] device                       */
  int64_t uniq_cap;
  int64_t K;                /* out: distinct rows                            */
  int32_t status;           /* out                                           */
  int32_t pad0;
  void* workspace;
  size_t workspace_bytes;
} mape_dedup_item;
size_t mape_dedup_batch_workspace_bytes(int32_t count);
int mape_dedup_batch(mape_dedup_item* items, int32_t count, void* workspace,
                     size_t workspace_bytes, void* stream);

/* a9 -- condition C1 (§3): ok[k] = 1 iff A g_k = 0 exactly.
 *   A [m x n] int32 (row-major, device), G [K x ldg] int8 (ldg a multiple of
 *   16, at most 4096).  *fail_count = rows with A g != 0.
 * Two exact implementations: when every A_ij fits in int8 and the rows are at
 * most 256 bytes, int8 dot products (dp4a) accumulated in int32, exact because
 * |sum| <= 127 * 127 * n < 2^31; otherwise A is compressed to its nonzeros
 * (CSR, built on the device in the workspace) and each row of G, staged once
 * in shared memory, is multiplied through them with int64 sums (the cost per
 * row is nnz(A), not m n).  The workspace holds the CSR of a dense A
 * (mape_kernel_test_workspace_bytes(m, n)).
 * Errors: INVALID_ARG, SHAPE (n or ldg above 4096), CAPACITY (workspace), CUDA.
 * Synchronous (returns the count). */
size_t mape_kernel_test_workspace_bytes(int32_t m, int32_t n);
int mape_kernel_test(const int32_t* A, int32_t m, int32_t n, const int8_t* G,
                     int64_t K, int32_t ldg, uint8_t* ok, int64_t* fail_count,
                     void* workspace, size_t workspace_bytes, void* stream);

/* a9 for many instances at once: item i is one mape_kernel_test call (its
 * own A, G, flags and workspace of mape_kernel_test_workspace_bytes(m, n))
 * and gets the same flags and fail_count.  Every A goes to compressed rows
 * in its workspace (two launches over the rows of all the A's and one scan
 * block per instance), then one launch tests the rows of all instances, a
 * warp per four rows (the compressed-row product, exact for every int32 A).
 * `workspace` holds the batch's tables
 * (mape_kernel_test_batch_workspace_bytes(count)).  Errors: INVALID_ARG,
 * SHAPE as mape_kernel_test for any item (before any device work),
 * CAPACITY, CUDA.  Synchronous. */
typedef struct {
  const int32_t* A;         /* [m x n] int32 device                          */
  int32_t m, n;
  const int8_t* G;          /* [K x ldg] int8 device                         */
  int64_t K;
  int32_t ldg, pad0;
  uint8_t* ok;              /* [K] out                                       */
  int64_t fail_count;       /* out                                           */
  void* workspace;
  size_t workspace_bytes;
} mape_kernel_test_item;
size_t mape_kernel_test_batch_workspace_bytes(int32_t count);
int mape_kernel_test_batch(mape_kernel_test_item* items, int32_t count,
                           void* workspace, size_t workspace_bytes,
                           void* stream);

/* a11 -- condition C3 within the set: keep[k] = 1 iff no other row h (with
 * valid[h] != 0) satisfies h ⊑ g_k or -h ⊑ g_k, where x ⊑ y iff
 * x_i y_i >= 0 and |x_i| <= |y_i| for all i (§1).  Rows with valid[k] == 0
 * are neither kept nor used (valid may be NULL: all valid).  The kept rows
 * are written, in their input order, to `out` (pitch ldg); *K_out = their
 * number.  G must hold distinct rows in canonical sign.  Synchronous. */
size_t mape_minimal_workspace_bytes(int64_t K, int32_t n);
int mape_minimal_filter(const int8_t* G, int64_t K, int32_t n, int32_t ldg,
                        const uint8_t* valid, uint8_t* keep, int8_t* out,
                        int64_t* K_out, void* workspace,
                        size_t workspace_bytes, void* stream);

/* a11 for many instances at once: item i is one mape_minimal_filter call
 * (its own rows, valid flags, keep flags, output and workspace of
 * mape_minimal_workspace_bytes(K, n)) and gets the same keep flags, output
 * and K_out.  Every kernel of the filter runs once over the rows, positions
 * or blocks of all instances; one dominance launch covers the pattern-list
 * blocks of all of them.  `workspace`:
 * mape_minimal_filter_batch_workspace_bytes(items, count).  Errors:
 * INVALID_ARG, SHAPE as mape_minimal_filter for any item (before any device
 * work), CAPACITY, CUDA.  Synchronous. */
typedef struct {
  const int8_t* G;          /* [K x ldg] distinct rows in canonical sign      */
  int64_t K;
  int32_t n, ldg;
  const uint8_t* valid;     /* optional [K]                                   */
  uint8_t* keep;            /* [K] out                                        */
  int8_t* out;              /* [K x ldg] out: the kept rows in input order    */
  int64_t K_out;            /* out                                            */
  void* workspace;
  size_t workspace_bytes;
} mape_minimal_item;
size_t mape_minimal_filter_batch_workspace_bytes(const mape_minimal_item* items,
                                                 int32_t count);
int mape_minimal_filter_batch(mape_minimal_item* items, int32_t count,
                              void* workspace, size_t workspace_bytes,
                              void* stream);

/* a12 -- per-direction coefficients for Algorithm 1 with
 * f = x^T Q x + c^T x + sum w_i x_i^4:
 *   a[k]  = g^T Q g            (int64, exact)
 *   q4[k] = sum_i w_i g_i^4    (int64, exact; 0 when w == NULL)
 * Q is given by its upper triangle including the diagonal as COO triplets
 * (q_row <= q_col), nnz entries.  Asynchronous. */
int mape_direction_coeffs(const int32_t* q_row, const int32_t* q_col,
                          const int32_t* q_val, int32_t nnz, const int32_t* w,
                          int32_t n, const int8_t* G, int64_t K, int32_t ldg,
                          int64_t* a, int64_t* q4, void* stream);

/* a12 for many instances at once: item i is one mape_direction_coeffs call
 * and gets the same a and q4; one launch, a warp per four directions of any
 * instance.  `workspace`: mape_direction_coeffs_batch_workspace_bytes(count).
 * Errors: INVALID_ARG, SHAPE as mape_direction_coeffs for any item, CAPACITY,
 * CUDA.  Asynchronous (the items are copied before the call returns). */
typedef struct {
  const int32_t* q_row;
  const int32_t* q_col;
  const int32_t* q_val;
  int32_t nnz, n;
  const int32_t* w;         /* NULL: no quartic term                         */
  const int8_t* G;
  int64_t K;
  int32_t ldg, pad0;
  int64_t* a;
  int64_t* q4;
} mape_coeffs_item;
size_t mape_direction_coeffs_batch_workspace_bytes(int32_t count);
int mape_direction_coeffs_batch(const mape_coeffs_item* items, int32_t count,
                                void* workspace, size_t workspace_bytes,
                                void* stream);

/* a13-a14 -- Algorithm 1 (§2) for S starts at once, with the direction set
 * ±G as test set.  One iteration, for every start s still active:
 *   r_s = 2 Q x_s + c;  for every k, sign e in {+1,-1}, lambda in
 *   [1, lambda_max(x_s, e g_k)] (the largest lambda keeping l <= x + lambda e g
 *   <= u), Delta f = lambda^2 a_k + lambda e g_k^T r_s + quartic terms (all
 *   int64); take the minimal Delta f, ties to the lower k, then +g, then the
 *   smaller lambda; if Delta f < 0 move x_s += lambda e g_k, else start s
 *   stops.  A x = b holds along the way because A g = 0.
 * Runs until every start stopped or max_iters iterations.
 *   X     [S x n] int32 in/out (must satisfy l <= x <= u)
 *   fval  [S] int64 out: f(x_s) at the end
 *   moves optional [S x moves_cap x 4] int64: (k, e, lambda, f after move)
 *   nmoves optional [S] int32: moves taken per start
 *   *iters_out (host): iterations run.  Errors: INVALID_ARG, BOUNDS (a start
 *   outside [l, u]), OVERFLOW (|Delta f| bound above 2^62), CUDA.
 * Synchronous. */
typedef struct {
  int32_t n, S;
  int64_t K;
  const int8_t* G; int32_t ldg;
  int32_t score_lanes;     /* lanes sharing a direction in the scoring pass:
                              1, 2, 4, 8, 16 or 32; 0 = autotuned per shape
                              (n, and K and S rounded up to powers of two,
                              quartic or not) on the call's own data.  Rows
                              are read as 16-byte pieces when ldg is a
                              multiple of 16 and G 16-byte aligned, else byte
                              by byte with one lane.  The results do not
                              depend on it. */
  const int64_t* a; const int64_t* q4;
  const int32_t* q_row; const int32_t* q_col; const int32_t* q_val; int32_t nnz;
  int32_t pad1;
  const int32_t* c; const int32_t* w; const int32_t* l; const int32_t* u;
  int32_t* X; int64_t* fval;
  int64_t* moves; int32_t* nmoves; int32_t moves_cap; int32_t pad2;
  int64_t max_iters;
  void* workspace; size_t workspace_bytes;
} mape_augment_args;
size_t mape_augment_workspace_bytes(int32_t n, int32_t S, int64_t K);
int mape_augment_run(const mape_augment_args* args, int64_t* iters_out,
                     void* stream);

/* a13-a14 for many instances at once (§3.3's multi-start augmentation over
 * a batch of instances): every item as in mape_augment_run, each with its
 * own directions, coefficients, objective, box, starts, outputs and
 * workspace of mape_augment_workspace_bytes.  One launch per iteration scores
 * the directions of every start of every instance and one applies the moves;
 * a chunk of 8 iterations (with a device iteration counter, so that an
 * instance stops at its own max_iters) is captured once as a CUDA graph and
 * replayed until every start of every instance has stopped (on the legacy
 * default stream, which cannot be captured, the chunk is launched directly).
 * The lane count of the scoring pass is the items' own when they all give the
 * same one, else the autotuned one of the item with the most row entries.
 * iters_out [count] (host): each item's mape_augment_run *iters_out.  Every
 * item's results (X, fval, moves, nmoves, iterations) are identical to its
 * own mape_augment_run.  `workspace` holds the batch's tables
 * (mape_augment_run_batch_workspace_bytes(count)).
 * done (optional) is called on the calling thread, once per item, as soon as
 * a chunk shows that the item has finished (every start stopped, or its
 * max_iters reached; items without starts or directions at once), with its
 * iteration count; from then on the batch no longer writes that item's
 * arrays (its X, fval, moves and nmoves may be read on another stream).
 * Errors: as mape_augment_run; BOUNDS if a start of any item lies outside its
 * box (no item then iterates); after an error done is not called for the
 * items not yet reported.  Synchronous. */
typedef void (*mape_augment_done_fn)(int32_t item, int64_t iters, void* ctx);
size_t mape_augment_run_batch_workspace_bytes(int32_t count);
int mape_augment_run_batch(const mape_augment_args* items, int32_t count,
                           int64_t* iters_out, void* workspace,
                           size_t workspace_bytes, void* stream,
                           mape_augment_done_fn done, void* done_ctx);

typedef struct {
  int32_t lanes;           /* chosen lanes per direction                     */
  int32_t candidates;      /* lane counts timed                              */
  int32_t cand_lanes[8];
  float probe_ms[8];       /* one scoring pass each, on the call's data      */
} mape_augment_tune_info;
/* The autotuned lane count of the scoring pass for a shape (n; K and S are
 * rounded up to powers of two), or STATE if none was tuned yet.
 * mape_autotune_clear forgets these choices too. */
int mape_augment_tune_lookup(int32_t n, int64_t K, int32_t S, int32_t quartic,
                             mape_augment_tune_info* out);

/* Eq. (4) (§3.3) -- initial feasible solutions of model (1): projected Adam
 * on ||A x - b||_2^2 + lambda3 sum_i (x_i - floor x_i)(ceil x_i - x_i) over
 * the box [l, u] from every start row of X (starts outside the box are
 * clipped into it first).  After every step whose number is a multiple of
 * `period` the rounded iterate (ties to even) is tested exactly, A round(x)
 * = b in int64 (the box holds by the projection), and, when it changed since
 * the start's previous collection in this call (the first collection of a
 * call always counts), appended to `sol` as n bytes round(x) - l (so u - l
 * must be at most 255).  FP32 CUDA-core arithmetic, one warp per start.
 * Continuing a run: pass X, M, V back with t0 = steps taken. */
typedef struct {
  int32_t n, m, P;
  int32_t pad0;
  const int32_t* A;        /* [m x n] int32                                  */
  const int64_t* b;        /* [m]                                            */
  const int32_t* l;        /* [n]                                            */
  const int32_t* u;        /* [n]                                            */
  float* X;                /* [P x n] in/out                                 */
  float* M;                /* [P x n] in/out, Adam first moment              */
  float* V;                /* [P x n] in/out, Adam second moment             */
  int32_t t0, T, period;
  float lambda3;           /* 0.1 in §4                                      */
  float lr, eps;
  double beta1, beta2;
  uint8_t* sol;            /* [sol_cap x lds] output rows round(x) - l        */
  int32_t lds;             /* row pitch in bytes, >= n                       */
  int32_t pad1;
  int64_t sol_cap;
  unsigned long long* sol_count;  /* device counter, appended to            */
  int32_t* flags;          /* device word, OR-ed: 1 = sol overflow           */
  float* dbg_f;            /* optional [P]: objective at the input point     */
  float* dbg_grad;         /* optional [P x n]: gradient at the input point  */
  void* workspace;
  size_t workspace_bytes;
} mape_init_args;
/* Errors: INVALID_ARG, SHAPE (n > 49152, or n + m too large for the warps'
 * shared memory), CAPACITY (workspace), CUDA.  Asynchronous. */
size_t mape_initial_solutions_workspace_bytes(int32_t n, int32_t m, int32_t T);
int mape_initial_solutions(const mape_init_args* args, void* stream);

/* Lemma 3.1, Theorem 3.2 -- a basis of Ker_Z(A) for a general A [m x n]
 * (full row rank, int32, row-major): unimodular integer column operations K
 * bring A to (H | 0); the last d = n - m columns of K are written to
 * B [n x d] (row-major).  reduce != 0 then applies the LLL reduction of
 * Appendix A (size reduction, exchange while ||B*_{i-1}||^2 > 2 ||B*_i||^2)
 * with double-precision Gram-Schmidt data.  A B = 0 is checked exactly.
 * Errors: INVALID_ARG (also: A not of full row rank), SHAPE (an intermediate
 * entry beyond 2^62 or a basis entry beyond int32), NUMERIC.  Host-only. */
int mape_kernel_basis(int32_t m, int32_t n, const int32_t* A, int32_t reduce, int32_t* B);

/* §3.4, Corollary 3.3 -- linear inequalities G x >= h (G [m2 x n], h [m2]):
 * writes the equality form of the instance with slack s = G x - h >= 0,
 *   A2 [(m+m2) x (n+m2)] = [A 0; G -I],  b2 = (b, h),
 *   l2 = (l, 0), u2 = (u, smax) with smax_k = max over the box of (G x)_k - h_k,
 *   B2 [(n+m2) x d] = [B; G B]  (a basis of Ker_Z(A2), with B's identity top),
 * all host arrays (row-major) owned by the caller.  The objective of the
 * extended instance is f of the first n coordinates (zero rows and columns
 * for the slacks).  Errors: INVALID_ARG, BOUNDS (some inequality holds
 * nowhere in the box), SHAPE (G B or smax beyond int32).  Host-only. */
int mape_inequality_extension(int32_t n, int32_t m, int32_t m2, const int32_t* A,
                              const int64_t* b, const int32_t* l, const int32_t* u,
                              const int32_t* G, const int64_t* h, const int32_t* B,
                              int32_t* A2, int64_t* b2, int32_t* l2, int32_t* u2,
                              int32_t* B2);

/* §3.4, Corollary 3.3 -- the objective and the points of the extended
 * instance of mape_inequality_extension:
 *   objective: Q2 [(n+m2) x (n+m2)] = [Q 0; 0 0], c2 = (c, 0), w2 = (w, 0)
 *     (w may be NULL, then w2 is not written): f of the original variables;
 *   points: for each of the S rows x of X [S x n], X2 [S x (n+m2)] = (x, s)
 *     with the slacks s = G x - h, so that x feasible for A x = b, G x >= h
 *     in the box maps to a point of the extended model (1).
 * Errors: INVALID_ARG, BOUNDS (some x violates G x >= h), SHAPE (a slack
 * beyond int32).  Host-only, host arrays owned by the caller. */
int mape_inequality_extension_objective(int32_t n, int32_t m2, const int32_t* Q, const int32_t* c,
                                        const int32_t* w, int32_t* Q2, int32_t* c2, int32_t* w2);
int mape_inequality_extension_points(int32_t n, int32_t m2, const int32_t* G, const int64_t* h,
                                     const int32_t* X, int32_t S, int32_t* X2);

/* ========================================================================== *
 * Instance handle (host pointers)                                             *
 * ========================================================================== */

typedef struct mape_instance* mape_handle;

/* Device memory hooks used by every handle created afterwards.
 * alloc(bytes, stream, ctx) returns a device pointer or NULL; free(ptr,
 * bytes, stream, ctx).  Passing NULLs restores the default: stream-ordered
 * allocation (cudaMallocFromPoolAsync / cudaFreeAsync) from a memory pool
 * per device that the library owns and that keeps freed memory reserved for
 * the next handle (no new page mappings when handles come and go). */
typedef void* (*mape_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*mape_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
int mape_set_allocator(mape_alloc_fn alloc_fn, mape_free_fn free_fn, void* ctx);

/* Returns the memory the current device's library pool holds beyond what
 * live handles use (cudaMemPoolTrimTo(pool, 0) after a device
 * synchronisation).  OK when the pool was never created. */
int mape_trim_memory(void);

typedef struct {
  int32_t n, m;
  const int32_t* Q;   /* [n x n] symmetric                                  */
  const int32_t* c;   /* [n]                                                */
  const int32_t* w;   /* [n] >= 0, or NULL: no quartic term                 */
} mape_problem;

/* Validates and uploads one instance.  A [m x n], b [m] int64, l, u [n],
 * B [n x d] (d = n - m) with A B = 0 checked on the device.
 * Errors: INVALID_ARG, SHAPE, BOUNDS, NOT_KERNEL_BASIS, OOM, CUDA. */
int mape_create_instance(const int32_t* A, const int64_t* b, const int32_t* l,
                         const int32_t* u, const mape_problem* f,
                         const int32_t* B, const mape_config* cfg,
                         void* stream, mape_handle* out);

/* Starts Algorithm 2 on the worker thread: P starts given either directly
 * (Z0 [P x d], G0 == NULL) or as samples to project (G0 [P x n], Z0 == NULL).
 * Z0 / G0 may be host or device pointers (unified addressing); they are
 * copied before the call returns.
 * The first call of a handle with G0 starts also forms the projection
 * W = B (B^T B)^{-1} (as mape_project_prepare; NUMERIC if B^T B is not
 * positive definite) and keeps it for later calls; calls with Z0 never need it.
 * Followed by dedup (a10), the kernel test (a9), the minimality filter (a11)
 * and the direction coefficients (a12).  Returns at once. */
int mape_extract_directions(mape_handle h, int32_t P, const float* Z0,
                            const float* G0);

/* Starts Algorithm 2 for `count` handles together (the paper has no batched
 * form; this is the interface a server uses to run uneven instances in one
 * launch): for handle i, P[i] starts Z0[i] or G0[i] as in
 * mape_extract_directions (Z0 or G0 may be NULL as a whole).  The extraction
 * steps of all handles run as one mape_extract_batch call per chunk of steps
 * (one CUDA graph of persistent launches, on the first handle's stream), each
 * chunk's candidates are merged into each handle's set on its own stream, and
 * the kernel test, minimality filter and coefficients of each handle then run
 * on its own worker thread and stream.  Every handle must be idle, and all
 * must share T, period and a BF16 precision (MAPE_PREC_BF16 or
 * MAPE_PREC_BF16X1, without MAPE_PREC_SPARSE_FWD): INVALID_ARG otherwise.
 * Returns at once; poll and wait on each handle as usual.  Each handle's
 * direction set equals that of its own mape_extract_directions. */
int mape_extract_directions_batch(mape_handle* hs, int32_t count, const int32_t* P,
                                  const float* const* Z0, const float* const* G0);

/* Starts Algorithm 1 from S starts X0 [S x n] (each must lie in S; host or
 * device pointer, copied before the call returns) with the current direction
 * set.  f_or_NULL replaces the objective (same n): the
 * direction set is reused for a new f (§1, reusability).  Returns at once. */
int mape_augment(mape_handle h, const int32_t* X0, int32_t S,
                 const mape_problem* f_or_NULL);

/* Starts Algorithm 1 for `count` handles together: handle i from S[i]
 * starts X0[i] (as in mape_augment, with each handle's current objective and
 * direction set).  The iterations of all handles run as
 * mape_augment_run_batch calls on the first handle's stream (the first
 * iteration alone, then the rest, as mape_augment does for one handle); each
 * handle then reads back its own best start.  Every handle must be idle, on
 * one device, with a direction set.  Returns at once; poll and wait on each
 * handle as usual.  Each handle's results (points, values, iteration counts)
 * equal those of its own mape_augment. */
int mape_augment_batch(mape_handle* hs, int32_t count, const int32_t* const* X0,
                       const int32_t* S);

#define MAPE_PHASE_IDLE       0
#define MAPE_PHASE_EXTRACTING 1
#define MAPE_PHASE_FILTERING  2
#define MAPE_PHASE_AUGMENTING 3
#define MAPE_PHASE_DONE       4
#define MAPE_PHASE_ERROR      5

typedef struct {
  int32_t phase;            /* MAPE_PHASE_*                                  */
  int32_t error;            /* status of the last finished job               */
  int64_t candidates;       /* rows collected by Algorithm 2                  */
  int64_t unique;           /* distinct rows                                  */
  int64_t kernel_failures;  /* rows with A g != 0 (always 0 unless corrupted) */
  int64_t directions;       /* rows kept after the minimality filter          */
  int64_t aug_iters;        /* Algorithm 1 iterations in the last augment     */
  int64_t best_f;           /* best f over the augmentation starts            */
  int32_t best_start;       /* which start reached best_f                     */
  int32_t pad0;
  double extract_ms, filter_ms, augment_ms;  /* stage wall times             */
  double first_improve_ms;  /* augment start -> first improving move found    */
} mape_status;

int mape_poll(mape_handle h, mape_status* st);          /* never blocks      */
int mape_wait(mape_handle h, int64_t timeout_ns);       /* TIMEOUT, no hang  */
int mape_cancel(mape_handle h);                          /* stops at next stage
                                                            boundary          */

/* Copies the direction set (K rows of n int32, sorted lexicographically) to
 * G [cap x n].  CAPACITY if cap < K (K is still set). */
int mape_get_directions(mape_handle h, int32_t* G, int64_t cap, int64_t* K);

/* The same rows as int8, the library's own storage type (every entry lies in
 * the box spans of C4, |g_i| <= 127): row k at G + k * ldg_out, n bytes each
 * (ldg_out >= n).  One strided device-to-host copy, no conversion; pinned
 * host memory makes it a single DMA.  CAPACITY if cap < K (K is still set);
 * INVALID_ARG if ldg_out < n. */
int mape_get_directions_i8(mape_handle h, int8_t* G, int64_t cap, int64_t ldg_out, int64_t* K);

/* Copies the best solution x [n] and f(x) of the last augment. */
int mape_get_solution(mape_handle h, int32_t* x, int64_t* fval);

/* Copies every start's final point X [S x n] and value fval [S]. */
int mape_get_solutions(mape_handle h, int32_t* X, int64_t* fval, int32_t S);

/* Eq. (4) on the handle's instance: P starts X0 [P x n] (host or device
 * pointer, copied; e.g. uniform in [l, u]), T steps of projected Adam with
 * lambda3 = 0.1 and the handle's Adam settings, collection every `period`
 * steps; the distinct exactly feasible points found are written to
 * X_out [cap x n] (sorted by the bytes round(x) - l) and counted in *S_out,
 * ready to be the starts of mape_augment (multi-start augmentation, §3.3).
 * CAPACITY if cap < *S_out.  Synchronous; the handle must be idle. */
int mape_find_initial_solutions(mape_handle h, int32_t P, const float* X0, int32_t T,
                                int32_t period, int32_t* X_out, int32_t cap,
                                int32_t* S_out);

void mape_destroy(mape_handle h);

/* ========================================================================== *
 * Request server: continuous batching of instances on one GPU                *
 * ========================================================================== */

/* Requests (an instance with its starts and augmentation starts) are copied
 * at submission and queued.  A scheduler thread admits them in arrival order
 * while one of `max_slots` slots is free and the device-memory estimate
 * (mape_request_bytes) of the running requests plus the next stays within
 * `mem_cap_bytes`.  An admitted request runs on its slot's own stream through
 * an instance handle: Algorithm 2 with dedup, kernel test and minimality
 * filter, then Algorithm 1 from its starts.  The running requests' kernels
 * overlap on the device; a request arriving while others run is admitted as
 * soon as a slot and memory free up.  Each request's result is independent of
 * what runs beside it.  (The paper has no server; this is an interface.) */
typedef struct mape_server* mape_server_h;

typedef struct {
  mape_config cfg;          /* hyper-parameters of every request             */
  size_t mem_cap_bytes;     /* admission budget of device memory             */
  int32_t max_slots;        /* requests on the device at once (1..256)       */
  int32_t keep_directions;  /* 1: keep each request's direction set on the
                               host for mape_server_result                  */
  int32_t batch_extraction; /* 1: the extraction of the requests admitted
                               together (whose handles are ready at the same
                               time) runs as one mape_extract_directions_batch
                               call, i.e. one graph of persistent launches per
                               chunk of steps for all of them; needs a BF16
                               precision.  Likewise the requests whose
                               direction sets are ready together start
                               Algorithm 1 as one mape_augment_batch call
                               (once no request is extracting, or the oldest
                               waiting one has waited 5 ms).  0: each
                               request's extraction and augmentation run on
                               its own slot stream                           */
  int32_t reserved;
} mape_server_config;

#define MAPE_REQ_QUEUED  0
#define MAPE_REQ_RUNNING 1
#define MAPE_REQ_DONE    2
#define MAPE_REQ_FAILED  3

typedef struct {
  int32_t state, error;       /* MAPE_REQ_*, status of a failed request    */
  int32_t n, m, P, pad0;
  int64_t directions;         /* size of the direction set                  */
  int64_t best_f;             /* best f over the augmentation starts        */
  int64_t aug_iters;
  size_t bytes;               /* admission estimate                         */
  /* server clock, milliseconds: submission, admission, end of extraction
   * (direction set ready), first improving move found, completion; time to
   * first improving direction = t_first_improve - t_submit, time to
   * termination = t_done - t_submit */
  double t_submit_ms, t_admit_ms, t_extracted_ms, t_first_improve_ms, t_done_ms;
} mape_request_info;

typedef struct {
  int64_t submitted, completed, failed, queued, running, peak_running;
  size_t mem_in_use, mem_peak, mem_cap;
} mape_server_stats;

/* Device bytes a request of these sizes holds while it runs (what the handle
 * allocates for the instance, its extraction and its augmentation), or 0 for
 * invalid sizes.  Host-only arithmetic. */
size_t mape_request_bytes(int32_t n, int32_t m, int32_t P, int32_t S, const mape_config* cfg);

/* Errors: INVALID_ARG, CUDA. */
int mape_server_create(const mape_server_config* cfg, mape_server_h* out);

/* Queues a request; arguments as mape_create_instance, mape_extract_directions
 * (Z0 [P x d] or G0 [P x n], host memory) and mape_augment (X0 [S x n]), all
 * copied before the call returns.  *id identifies the request.
 * Errors: INVALID_ARG, SHAPE, OOM (the request alone exceeds the memory cap,
 * so it could never be admitted). */
int mape_server_submit(mape_server_h s, const int32_t* A, const int64_t* b,
                       const int32_t* l, const int32_t* u, const mape_problem* f,
                       const int32_t* B, int32_t P, const float* Z0,
                       const float* G0, const int32_t* X0, int32_t S,
                       uint64_t* id);

int mape_server_poll(mape_server_h s, uint64_t id, mape_request_info* info); /* never blocks */
int mape_server_wait(mape_server_h s, uint64_t id, int64_t timeout_ns);      /* TIMEOUT, or the
                                                                                request's status */
int mape_server_wait_all(mape_server_h s, int64_t timeout_ns);               /* queue empty and
                                                                                nothing running */

/* Best x [n] and f of a finished request; with keep_directions, K and (if
 * G != NULL) the direction set as int8 rows G [cap x n], sorted
 * lexicographically.  CAPACITY if cap < K. */
int mape_server_result(mape_server_h s, uint64_t id, int32_t* x, int64_t* fval,
                       int8_t* G, int64_t cap, int64_t* K);

/* Forgets a finished request (its host results). */
int mape_server_release(mape_server_h s, uint64_t id);

int mape_server_get_stats(mape_server_h s, mape_server_stats* st);

/* Waits (up to 10 minutes) for the running requests, then stops. */
void mape_server_destroy(mape_server_h s);

/* Launch timing, for measurement (no counterpart in the paper): while on,
 * every launch of the extraction kernels below is bracketed by a pair of CUDA
 * events on its stream; mape_launch_timing_read synchronises on them and
 * returns, per kind, the summed milliseconds between each pair and the number
 * of launches since timing was switched on (or last read: reading clears the
 * pending pairs, not the sums).  mape_launch_timing(enable) switches it and
 * clears everything.  The events add a little time around each launch, so
 * time a region either with or without it. */
#define MAPE_TIMED_STREAM_FWD     0   /* streamed forward + map kernel       */
#define MAPE_TIMED_STREAM_COLLECT 1   /* streamed collection kernel          */
#define MAPE_TIMED_STREAM_GRAD    2   /* streamed gradient + Adam kernel     */
#define MAPE_TIMED_RESIDENT       3   /* resident fused kernel (T steps)     */
#define MAPE_TIMED_KINDS          4
int mape_launch_timing(int32_t enable);
int mape_launch_timing_read(double* ms /* [MAPE_TIMED_KINDS] */,
                            int64_t* launches /* [MAPE_TIMED_KINDS] */);

/* Tensor-core instruction cost on this GPU, for measurement (no counterpart
 * in the paper): one thread issues `chain` tcgen05.mma instructions
 * (cta_group::1; kind 0: kind::f16 with BF16 operands, K = 16; kind 1:
 * kind::f8f6f4 with e4m3 operands, K = 32) of shape M x N (M 64 or 128,
 * N 16..256 in steps of 16) into 1 or 2 TMEM accumulators; *issue_cycles and
 * *total_cycles are SM cycles per instruction from the first issue to the last
 * issue and to the completion of the chain.  Synchronous on the legacy
 * default stream; allocates 24 bytes of device memory.  Errors: INVALID_ARG,
 * CUDA, TIMEOUT (the completion wait gave up after 2 s). */
int mape_mma_issue_probe(int32_t kind, int32_t M, int32_t N, int32_t accumulators, int32_t chain,
                         double* issue_cycles, double* total_cycles);

/* Version string of the library build. */
const char* mape_version(void);

/* Text of the last CUDA runtime error recorded by any call, or of the last
 * argument error that a call explained there (or ""). */
const char* mape_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all handles); the difference across a region counts its launches. */
unsigned long long mape_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MAPE_H_ */
