/*
 * cpgrad -- fast all-mode CP gradients and CP_ALS on NVIDIA GB300 (sm_103a).
 *
 * The library computes the CP gradient of a dense N-way tensor Y
 * (eq. 2.13, product term; Section 2.2):
 *
 *     G^(n) = Y_(n) (A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1)),
 *
 * for one mode or for every mode, following Algorithm 2 (Section 3.3): the
 * tensor is viewed, without moving data, as the J x K matrix
 * reshape(Y, [J_k, K_k]) (eq. 2.3) at a split k, one leading contraction on
 * each side of k (Algorithm 2, steps 4 and 7) streams Y from memory, and all
 * other modes follow from the much smaller partial tensors R^(n), L^(n)
 * (eqs. 3.19-3.22, steps 11, 15, 19, 20).  No mode-n unfolding is ever formed.
 * On top of it sits the fast CP_ALS sweep of Section 4 (update rule eq. 2.14).
 *
 * Conventions shared by every entry point
 *  - Tensor layout: vec(Y) with mode 1 fastest (column-major, eq. 2.1).  Y is a
 *    DEVICE pointer to prod(I) elements.
 *  - Modes are 0-based in this API (the paper is 1-based): n in [0, N).
 *  - Factor A^(n) and gradient G^(n) are I_n x R column-major matrices
 *    (leading dimension I_n), DEVICE pointers.  `A` and `G` are HOST arrays
 *    of N such device pointers.
 *  - Element type: double when opts->precision == CPG_FP64, float otherwise
 *    (Y, A, G alike).  lambda and fit are always double.
 *  - The caller owns all memory.  The library never allocates device memory:
 *    every call takes a caller-provided device workspace of at least
 *    cpg_workspace_size(...) bytes (opts->workspace, 256-byte aligned), whose
 *    first 256 bytes hold the device status word (cpg_workspace_init clears it).
 *  - Calls are asynchronous on opts->stream (a cudaStream_t; NULL = legacy
 *    default stream).  The returned status covers argument checks and launch
 *    errors.  Conditions found on the device (a singular normal-equation
 *    matrix in CP_ALS, a bounded wait that expired) are recorded in a status
 *    word inside the workspace; cpg_device_status() synchronizes the stream
 *    and returns and clears it.
 *  - Argument errors (return CPG_ERR_ARG): N < 2 or N > CPG_MAX_ORDER, any
 *    I_n < 1, R < 1 or R > CPG_MAX_RANK, a NULL pointer where one is
 *    required, a mode n out of range, split not in {0} U [1, N-1], an unknown
 *    precision.  prod(I) overflowing int64 returns CPG_ERR_SHAPE.  A workspace
 *    that is NULL or too small returns CPG_ERR_WORKSPACE.  A precision that
 *    has no kernel for the call returns CPG_ERR_UNSUPPORTED.  Nothing is
 *    launched when a call returns an error.
 */
#ifndef CPGRAD_H
#define CPGRAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPG_MAX_ORDER 16
#define CPG_MAX_RANK 256

typedef enum {
  CPG_OK = 0,
  CPG_ERR_ARG = 1,
  CPG_ERR_SHAPE = 2,
  CPG_ERR_WORKSPACE = 3,
  CPG_ERR_SINGULAR = 4,
  CPG_ERR_CUDA = 5,
  CPG_ERR_TIMEOUT = 6,
  CPG_ERR_UNSUPPORTED = 7
} cpg_status;

/* Arithmetic of the leading contraction (Algorithm 2, steps 4 and 7), the
 * part that streams Y.  Everything after it runs in FP32 (FP64 for
 * CPG_FP64).  The CP_ALS normal equations run in double-float arithmetic
 * (pairs of floats, about 48 significant bits) for FP32 data and in FP64 for
 * CPG_FP64.  The split BF16 forms split each FP32 value into BF16 limbs
 * (round to nearest) and keep the products of total limb order below the
 * limb count (Henry, Tang and Heinecke, 2019); each tensor-core stage's
 * partial sums are added into FP32 running sums with round-to-nearest adds.
 * The iterative sweeps (cp_als_iter, cp_ntf_iter, cp_als_batched) accept
 * CPG_FP32, CPG_TF32X3, CPG_BF16X6 and CPG_FP64 only (CPG_ERR_UNSUPPORTED
 * otherwise): one and two BF16 limbs carry about 9 and 17 significant bits,
 * an error each sweep's solve would carry into the factors. */
typedef enum {
  CPG_FP32 = 0,    /* FP32 CUDA-core FMA, FP32 accumulation                        */
  CPG_TF32X3 = 1,  /* 3-term split TF32 products on tcgen05, FP32 accumulation    */
  CPG_BF16X3 = 2,  /* two BF16 limbs, 3 products on tcgen05 (gradient calls only) */
  CPG_BF16 = 3,    /* one BF16 limb, 1 product on tcgen05 (gradient calls only)   */
  CPG_FP64 = 4,    /* FP64 tensor and factors, FP64 CUDA-core FMA                 */
  CPG_BF16X6 = 5   /* three BF16 limbs, 6 products on tcgen05                     */
} cpg_precision;

typedef struct {
  int precision;          /* cpg_precision                                      */
  int split;              /* k = number of leading modes in J; 0 = n* (Alg. 2 step 1) */
  void* workspace;        /* device scratch, >= cpg_workspace_size() bytes       */
  size_t workspace_bytes;
  void* stream;           /* cudaStream_t; NULL = legacy default stream          */
} cpg_opts;

/* Which call a workspace is sized for (CPG_CALL_GRADIENT_TUNE:
 * cpg_autotune_gradient, the largest of its candidate plans). */
typedef enum {
  CPG_CALL_GRADIENT_ALL = 0,
  CPG_CALL_GRADIENT_MODE = 1,
  CPG_CALL_ALS = 2,
  CPG_CALL_GRADIENT_TUNE = 3,
  CPG_CALL_GRADIENT_FULL = 4,  /* cp_gradient_full and cp_gradient_step */
  CPG_CALL_NTF = 5,            /* cp_ntf_iter */
  CPG_CALL_ALS_TUNE = 6        /* cpg_autotune_als */
} cpg_call;

/* n* = max{n : J_n <= K_n} of Algorithm 2 step 1, 1-based count of leading
 * modes, clamped into [1, N-1] (when I_1 > I_2...I_N no n qualifies and 1 is
 * returned).  Host-only; returns 0 on invalid arguments. */
int cpg_split_point(const int64_t* I, int N);

/* Bytes of device workspace that `call` needs for this shape, rank and
 * options (opts->precision and opts->split are read; NULL opts = defaults).
 * Host-only.  Returns 0 on invalid arguments.
 * When the column pitch of reshape(Y, [J_k, K_k]) (J_k times the element
 * size) is not a multiple of 16 bytes, the sizes for CP_ALS (CPG_CALL_ALS,
 * CPG_CALL_NTF) and for a gradient that reads Y twice include a copy of Y
 * with the pitch rounded up to 16 bytes: those calls copy Y once and stream
 * the copy with TMA tiles.  Given a smaller workspace that still holds
 * everything else, they skip the copy and stream Y itself with element copies
 * (same results, about half the bandwidth). */
size_t cpg_workspace_size(const int64_t* I, int N, int R, const cpg_opts* opts, int call);

/* All-mode CP gradient, Algorithm 2 (Section 3.3): G[n] <- Y_(n) KR_{m != n}
 * for every n in [0, N).  The two leading contractions (steps 4 and 7) are
 * computed from one pass over Y (both from each tile) or from two, one per
 * side: the measured plan of cpg_autotune_gradient when one is recorded,
 * else the planner's, which fuses the CUDA-core passes only at R <= 4 and the
 * tensor-core passes for BF16 and BF16x3 at R <= 32, when the partial sums of
 * the fused pass stay below a fifth of Y's size.  The other modes follow from
 * R^(n) and L^(n) (steps 11, 15, 19, 20).  G[n] are overwritten. */
cpg_status cp_gradient_all(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                           void* const* G, const cpg_opts* opts);

/* A plan of the all-mode gradient: the split k (number of leading modes in
 * J, Algorithm 2 step 1) and whether steps 4 and 7 share one pass over Y. */
typedef struct {
  int split;       /* 1 <= split <= N-1                                   */
  int fused;       /* 1: one pass computes steps 4 and 7; 0: two passes   */
  float ms;        /* measured milliseconds per call (autotune only)      */
  int candidates;  /* plans timed (autotune only)                         */
} cpg_gradient_plan;

/* Measured choice of the all-mode gradient's plan.  The paper picks the split
 * n* by a cost model (Algorithm 2 step 1, Section 3.1); here every candidate
 * is timed on the caller's data instead: each split k in [1, N-1] (or only
 * opts->split when it is nonzero), as two single-side passes and, where the
 * precision has one and its partial sums stay below the tensor's size, as one
 * fused pass.  Each candidate runs once untimed, then `reps` times (1..1000)
 * between CUDA events on opts->stream; the call synchronizes that stream, so
 * it cannot be captured in a CUDA graph.  The fastest plan is recorded for
 * this device, precision, requested split, rank and shape (process-wide,
 * thread-safe) and written to *chosen (may be NULL).  G receives the gradient.
 * Later cp_gradient_all / cp_gradient_all_noalloc calls with the same key run
 * the recorded plan whenever their workspace holds it (cpg_workspace_size
 * accounts for it), else the planner's.  Every plan computes the same
 * gradient up to rounding.  The workspace must hold
 * cpg_workspace_size(..., CPG_CALL_GRADIENT_TUNE) bytes, else
 * CPG_ERR_WORKSPACE; argument errors as for cp_gradient_all. */
cpg_status cpg_autotune_gradient(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                                 void* const* G, const cpg_opts* opts, int reps, cpg_gradient_plan* chosen);

/* 1 and *plan (split, fused) when a measured plan is recorded for this shape,
 * rank and opts (precision, split, current device); 0 otherwise.  Host-only. */
int cpg_gradient_plan_query(const int64_t* I, int N, int R, const cpg_opts* opts, cpg_gradient_plan* plan);

/* Records *plan as the measured plan for this shape, rank and opts
 * (precision, split, current device), as cpg_autotune_gradient would: a plan
 * kept from an earlier run, or one a caller wants to pin.  Host-only.
 * CPG_ERR_ARG for a split outside [1, N-1] (or other than a nonzero
 * opts->split), CPG_ERR_UNSUPPORTED for a fused plan the precision has no
 * fused pass for; shape errors as for cp_gradient_all. */
cpg_status cpg_gradient_plan_set(const int64_t* I, int N, int R, const cpg_opts* opts,
                                 const cpg_gradient_plan* plan);

/* Forgets every recorded plan (gradient plans and CP_ALS splits). */
void cpg_autotune_clear(void);

/* The split of a CP_ALS sweep: k leading modes, update order k-1, ..., 0,
 * k, ..., N-1 (Section 4 with n* replaced by k). */
typedef struct {
  int split;       /* 1 <= split <= N-1                              */
  float ms;        /* measured milliseconds per sweep (autotune only) */
  int candidates;  /* splits timed (autotune only)                    */
} cpg_als_plan;

/* Splits cpg_autotune_als times, cheapest modelled first: opts->split alone
 * when nonzero, else n* (Algorithm 2 step 1) and every k in [1, N-1] whose
 * modelled sweep cost is within 1.25x of the cheapest.  The model counts the elements a sweep moves: two
 * reads of Y (the same for every k), the Khatri-Rao operands of the two
 * passes, and twice (written, read) every partial result R^(m), m <= k, and
 * L^(m), m > k, of the recursions (steps 11 and 15 of Algorithm 2), which
 * are also the sizes Table 4.1's multiplication counts sum.  Writes up to
 * `cap` splits to `splits` (may be NULL) and returns how many there are;
 * 0 on invalid arguments.  Host-only. */
int cpg_als_candidates(const int64_t* I, int N, int R, const cpg_opts* opts, int* splits, int cap);

/* Measured choice of the CP_ALS split.  Each candidate of cpg_als_candidates
 * runs one untimed sweep, then `reps` sweeps (1..1000) between CUDA events on
 * opts->stream, each from the caller's starting A and lambda, which are saved
 * in the workspace first and restored after every run: on return A and lambda
 * hold their entry values.  The call synchronizes the stream, so it cannot be
 * captured in a CUDA graph.  The fastest split is recorded for this device,
 * precision, requested split, rank and shape (process-wide, thread-safe) and
 * written to *chosen (may be NULL).  Later cp_als_iter and cp_ntf_iter calls
 * with opts->split == 0 and the same key run the recorded split whenever
 * their workspace holds it (cpg_workspace_size accounts for it; so do the
 * members of cp_als_batched), else n*.  A candidate whose plan cannot run
 * at this size (refused before any launch) is skipped; CPG_ERR_UNSUPPORTED
 * when none can.  Workspace: cpg_workspace_size(..., CPG_CALL_ALS_TUNE)
 * bytes, else CPG_ERR_WORKSPACE; argument and precision errors as for
 * cp_als_iter. */
cpg_status cpg_autotune_als(const void* Y, const int64_t* I, int N, void* const* A, double* lambda, int R,
                            const cpg_opts* opts, int reps, cpg_als_plan* chosen);

/* 1 and *plan (split) when a measured CP_ALS split is recorded for this
 * shape, rank and opts (precision, split, current device); 0 otherwise.
 * Host-only. */
int cpg_als_plan_query(const int64_t* I, int N, int R, const cpg_opts* opts, cpg_als_plan* plan);

/* Records plan->split as the measured CP_ALS split for this shape, rank and
 * opts, as cpg_autotune_als would.  Host-only; errors as for
 * cpg_gradient_plan_set. */
cpg_status cpg_als_plan_set(const int64_t* I, int N, int R, const cpg_opts* opts, const cpg_als_plan* plan);

/* Single-mode CP gradient, Section 3.2: G^(n) via the right-to-left route
 * (eqs. 3.7, 3.10, 3.12) when J_n <= K_{n-1}, else the left-to-right route
 * (eqs. 3.8, 3.9, 3.16).  Gn (I_n x R) is overwritten. */
cpg_status cp_gradient_mode(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                            int n, void* Gn, const cpg_opts* opts);

/* `iters` sweeps of the fast CP_ALS of Section 4 with update rule eq. 2.14.
 * Mode order per sweep (0-based): k-1, k-2, ..., 0, k, ..., N-1, with k =
 * opts->split, else the split cpg_autotune_als recorded, else n*.
 * Each update solves A^(n) V = G^(n), V = Hadamard_{m != n} A^(m)T A^(m)
 * (Gauss-Jordan inverse of V in double-float arithmetic for FP32 data, FP64
 * Cholesky for FP64 data), then normalises the columns: lambda_r =
 * ||a_r^(n)||, a_r^(n) /= lambda_r.  R <= 64 (the gradient calls take up to CPG_MAX_RANK;
 * a larger R here returns CPG_ERR_UNSUPPORTED).  A[n] (device, I_n x R) and lambda (device, R
 * doubles) are updated in place; A on entry is the starting point.
 * fit (device, `iters` doubles, may be NULL) receives after each sweep
 * fit = 1 - ||Y - Yhat||_F / ||Y||_F computed from R x R quantities.
 * A V that is not positive definite leaves that mode unchanged and records
 * CPG_ERR_SINGULAR in the device status word. */
cpg_status cp_als_iter(const void* Y, const int64_t* I, int N, void* const* A, double* lambda, int R,
                       int iters, double* fit, const cpg_opts* opts);

/* Cost gradient of eq. 2.13 for every mode, with its model term:
 *     G[n] <- Y_(n) KR - A^(n) Gamma^(n),  Gamma^(n) = Hadamard_{m != n} A^(m)T A^(m),
 * i.e. E_(n) KR for the residual E = Y - [[A]] without forming E.  The
 * derivative of D = ||Y - Yhat||^2 (eq. 2.12) is -2 G[n].  Y_(n) KR comes from
 * Algorithm 2 (the plan of cp_gradient_all, measured when tuned); Gamma^(n) and
 * A^(n) Gamma^(n) are formed in FP64.  Workspace: cpg_workspace_size(...,
 * CPG_CALL_GRADIENT_FULL).  Errors as for cp_gradient_all. */
cpg_status cp_gradient_full(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                            void* const* G, const cpg_opts* opts);

/* One all-at-once first-order step (eq. 2.15): G as cp_gradient_full at the
 * current factors (every mode's gradient before any factor changes), then
 * A[n] <- A[n] + eta G[n] for every n (a step of eta / 2 along -dD/da).
 * A (device, in place) and G (device, out) as in cp_gradient_full; eta must
 * not be NaN (CPG_ERR_ARG). */
cpg_status cp_gradient_step(const void* Y, const int64_t* I, int N, void* const* A, int R, double eta,
                            void* const* G, const cpg_opts* opts);

/* `iters` sweeps of multiplicative nonnegative CP updates (eq. 2.18) in the
 * fast CP_ALS order of Section 4 (modes k-1, ..., 0, then k, ..., N-1, the
 * recursions using the factors just updated):
 *     A^(n) <- A^(n) * (Y_(n) KR) / (A^(n) Gamma^(n))   elementwise,
 * an entry whose denominator is not positive left as is; no normalisation.
 * Meant for nonnegative Y and A (they then stay nonnegative).  fit (device,
 * `iters` doubles, may be NULL) receives 1 - ||Y - Yhat|| / ||Y|| after each
 * sweep, from R x R quantities.  The FP32 path forms Y_(n) KR in FP32 and the
 * R x R products in FP64.  Workspace: cpg_workspace_size(..., CPG_CALL_NTF);
 * R <= 64; argument errors as for cp_als_iter (no lambda). */
cpg_status cp_ntf_iter(const void* Y, const int64_t* I, int N, void* const* A, int R, int iters, double* fit,
                       const cpg_opts* opts);

/* One member of a batched CP_ALS call.  Y, A[n], lambda and fit are device
 * buffers as in cp_als_iter; I and A are host arrays of N entries that are
 * read during the call only. */
typedef struct {
  const void* Y;     /* vec(Y) (eq. 2.1), FP32 (FP64 when precision is CPG_FP64) */
  int N;             /* order, 2 <= N <= CPG_MAX_ORDER                            */
  const int64_t* I;  /* host, [N] mode sizes                                      */
  void* const* A;    /* host, [N] device factors, I_n x R column-major, in place  */
  double* lambda;    /* device, [R]                                               */
  int R;             /* rank, 1 <= R <= 64                                        */
  double* fit;       /* device, [iters] fit after each sweep, or NULL             */
} cpg_tensor_desc;

/* Workspace bytes for cp_als_batched over these members (opts->precision and
 * opts->split are read; split applies to every member, 0 = each member's own
 * n*).  Host-only.  Returns 0 on invalid arguments. */
size_t cpg_workspace_size_batched(int B, const cpg_tensor_desc* descs, const cpg_opts* opts);

/* `iters` fast CP_ALS sweeps (as cp_als_iter) on each of B independent
 * tensors of any order, shape and rank.  The paper decomposes one tensor at a
 * time; batching many small problems is this library's extension of it.
 *  - Members run concurrently on a pool of streams owned by the library
 *    (largest members first, each to the least-loaded stream), forked from
 *    and joined back into opts->stream by events: the whole batch is ordered
 *    after earlier work on opts->stream and before later work on it, so
 *    capturing one call on opts->stream into a CUDA graph captures the batch.
 *  - Each member uses its own slice of opts->workspace; device errors of all
 *    members go to the one status word at the start of the workspace
 *    (cpg_device_status).
 *  - Argument errors of any member (as for cp_als_iter) return before
 *    anything is launched.
 * Results are bit-identical to B separate cp_als_iter calls. */
cpg_status cp_als_batched(int B, const cpg_tensor_desc* descs, int iters, const cpg_opts* opts);

/* Clears the device status word at the start of opts->workspace (stream
 * ordered).  Call once on a new workspace before its first use; the status
 * word is otherwise left as the device wrote it. */
cpg_status cpg_workspace_init(const cpg_opts* opts);

/* Synchronizes opts->stream, returns the device status word recorded since the
 * last call (CPG_OK if none) and clears it. */
cpg_status cpg_device_status(const cpg_opts* opts);

/* Failure-detection self-test (the paper has no counterpart).  Launches, on
 * opts->stream, one CTA whose mbarrier wait can never complete (nothing
 * arrives on the barrier), bounded by `polls` polls (1 .. 2^24) exactly as
 * every wait in this library's kernels is.  On expiry the CTA records
 * CPG_ERR_TIMEOUT in the status word at the start of opts->workspace and
 * returns: no fault, no hang, the context stays usable, and
 * cpg_device_status() reports the timeout.  CPG_ERR_ARG for a NULL workspace,
 * one smaller than 256 bytes, or polls out of range. */
cpg_status cpg_selftest_timeout(const cpg_opts* opts, unsigned polls);

/* Static description of a status code. */
const char* cpg_status_str(int status);

/* Kernel launches issued by this library on the calling thread since the
 * last reset (counts what the host enqueued; for benchmarks). */
uint64_t cpg_launch_count(int reset);

/* Benchmark instrumentation.  While enabled, launches are bracketed by two
 * CUDA events recorded on their own stream (at most 4096 launches are kept):
 * enable = 1 records the leading contraction (Algorithm 2 steps 4 and 7, the
 * kernel that streams Y), enable = 2 records every kernel of the library.
 * A nonzero enable creates the events on first use and starts a new record;
 * 0 stops recording.  Returns CPG_OK or CPG_ERR_CUDA.
 * Not thread-safe: one recording thread at a time. */
int cpg_profile_lead(int enable);

/* Kinds of recorded launches (cpg_profile_read). */
#define CPG_KIND_LEAD_R 1       /* leading pass, step 4 only                    */
#define CPG_KIND_LEAD_L 2       /* leading pass, step 7 only                    */
#define CPG_KIND_LEAD_FUSED 3   /* leading pass, steps 4 and 7 from one read    */
#define CPG_KIND_CHAIN 10       /* finishing contraction or recursion           */
#define CPG_KIND_MODE 11        /* CP_ALS mode, FP32 data: G and the update     */
#define CPG_KIND_GRAM 12        /* Gram matrices                                */
#define CPG_KIND_KRON 13        /* Kronecker vector of a run of modes           */
#define CPG_KIND_NORM 14        /* ||Y||^2                                      */
#define CPG_KIND_UPDATE 15      /* CP_ALS update (FP64 data), NTF update        */
#define CPG_KIND_MODEL_TERM 16  /* model term of eq. 2.13, step of eq. 2.15     */
#define CPG_KIND_ROWS 17        /* Khatri-Rao rows of a leading pass (eq. 3.9 / 3.10), once per pass */
#define CPG_KIND_PITCH 18       /* copy of Y_(1:k) with a 16-byte column pitch  */

/* Waits for and returns the recorded launch durations in milliseconds
 * (ms[i]) and each launch's kind (sides[i], CPG_KIND_*), at most `max`
 * entries in launch order, then clears the record.  Either array may be
 * NULL.  Returns the number of entries, or -1 on a CUDA error. */
int cpg_profile_read(float* ms, int* sides, int max);

/* Size of the fixed device scratch array used by cp_gradient_all_noalloc
 * (64 MiB, held by every GPU that loads the library until the process exits). */
#define CPG_NOALLOC_WORKSPACE_BYTES (64u << 20)

/* All-mode CP gradient without any device allocation, for callers that cannot
 * call cudaMalloc: for example a plugin inside a host application that owns
 * every device allocation through its own pool, or latency-critical code that
 * must not allocate after start-up.  The paper has no counterpart; this is a
 * calling convention of this library.
 *
 * Same computation and arguments as cp_gradient_all (Y, A, G are caller
 * device buffers), but the scratch comes from a fixed array of
 * CPG_NOALLOC_WORKSPACE_BYTES inside the library instead of opts->workspace.
 * precision and split are as in cpg_opts; stream is a cudaStream_t (NULL =
 * legacy default stream).
 *  - The argument errors of cp_gradient_all come first, in its order.  Then
 *    CPG_ERR_WORKSPACE when the plan the call would run with that much room
 *    (less the optional pitched copy of Y: without room for it the gradient
 *    streams Y itself) exceeds CPG_NOALLOC_WORKSPACE_BYTES.  Nothing is
 *    launched on an error.
 *  - The first call on a device looks up the array's device address (with
 *    that device current), clears its device status word synchronously and
 *    caches the address (thread-safe); make that first call, or one of
 *    cpg_noalloc_scratch, before any stream capture.  The cached address is
 *    not valid after cudaDeviceReset.
 *  - Device-side conditions (a bounded wait that expired) are recorded in the
 *    status word at the start of the array and kept until read: pass the
 *    address from cpg_noalloc_scratch as opts->workspace to cpg_device_status.
 *  - Every call shares the one array and leaves its contents behind.  Calls
 *    that overlap on the GPU (different streams or threads) race on it;
 *    calls on one stream are ordered.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
cpg_status cp_gradient_all_noalloc(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                                   void* const* G, int precision, int split, void* stream);

/* Device address (*ptr) and size (*bytes, may be NULL) of the fixed scratch
 * array of cp_gradient_all_noalloc on the current device, set up as that
 * call's first use on the device does.  With it a caller reads the array's
 * device status word (cpg_device_status with opts->workspace = *ptr), or runs
 * the bounded-wait self-test on it.  The paper has no counterpart.
 * CPG_ERR_ARG for a NULL ptr, CPG_ERR_CUDA if the lookup fails. */
cpg_status cpg_noalloc_scratch(void** ptr, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* CPGRAD_H */
