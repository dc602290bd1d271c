/*
 * lpb.h -- C ABI of liblpb, a batched linear-program solver for one GB300 GPU.
 *
 * Problem (Section 3, Eq. 1-3 of Gurung & Ray, "Solving Batched Linear Programs
 * on GPU and Multicore CPU"): for every LP k of a batch
 *
 *     maximize  c^T x   subject to  A x <= b,  x >= 0,         A is m_k x n_k,
 *
 * and, as a closed-form special case (Section 6, Eq. 8), the support function
 * of a hyperbox, maximize c^T x subject to l <= x <= u.
 *
 * Conventions shared by every call:
 *   - Pointers documented as "device" point to memory of the handle's GPU and
 *     are owned by the caller; the library never frees or keeps them past the
 *     call.  Calls are asynchronous on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) and return before the GPU work finishes.
 *   - The library allocates device memory only in lpb_create (a few bytes of
 *     counters and an error word).  All scratch comes from the caller's
 *     workspace `ws` of at least lpb_workspace_size() bytes, 256-byte aligned.
 *   - The return value (lpb_err) reports host-side validation and CUDA launch
 *     errors only.  Mathematical outcomes (optimal, infeasible, unbounded, ...)
 *     are per-LP lpb_status values written to result->status and are never an
 *     error.  Faults detected inside kernels (a size outside the declared
 *     bounds, an exhausted workspace) are recorded in the handle's device
 *     error word and reported by lpb_sync_error(), which synchronises.
 *   - No call traps, asserts or spins without bound on the device.
 */
#ifndef LPB_H_
#define LPB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-LP outcome (Section 3.1: the halt conditions "optimal" and "unbounded";
 * Section 3: the auxiliary-LP optimum is non-zero -> "infeasible"). */
typedef enum {
  LPB_OPTIMAL = 0,
  LPB_INFEASIBLE = 1,
  LPB_UNBOUNDED = 2,
  LPB_ITER_LIMIT = 3,   /* the pivot cap was reached */
  LPB_NUMERIC = 4,      /* NaN/Inf in the data, or a numerical breakdown */
  LPB_BAD_SIZE = 5      /* m or n outside 1..max_m / 1..max_n */
} lpb_status;

/* Per-call error codes. */
typedef enum {
  LPB_OK = 0,
  LPB_EINVAL = -1,        /* a NULL pointer, a negative count, bad options */
  LPB_ENOMEM = -2,        /* workspace smaller than lpb_workspace_size() */
  LPB_ECUDA = -3,         /* a CUDA runtime call failed */
  LPB_EUNSUPPORTED = -4,  /* a size or mode this build does not handle */
  LPB_EDEVICE = -5        /* a kernel recorded a fault in the device error word */
} lpb_err;

/* Arithmetic of the simplex tableau. */
typedef enum {
  LPB_FP64 = 0,         /* FP64 tableau throughout */
  LPB_FP32_REFINE = 1,  /* FP32 tableau; FP64 refinement, verification and FP64 re-solve */
  LPB_FP32 = 2          /* FP32 tableau, results converted to FP64 unrefined */
} lpb_precision;

typedef enum { LPB_DTYPE_F32 = 0, LPB_DTYPE_F64 = 1 } lpb_dtype;

/* A packed batch.  LP k has m[k] rows and n[k] structural variables; its
 * A is m[k] x n[k] row-major at element offset a_off[k] of A, its b has m[k]
 * elements at b_off[k] of b, its c has n[k] elements at c_off[k] of c.
 * m, n, a_off, b_off, c_off, A, b, c are device pointers.  max_m and max_n are
 * HOST values bounding every m[k] and n[k]; LPs outside them get LPB_BAD_SIZE.
 * dtype (lpb_dtype) applies to A, b and c.  min_m and min_n are optional HOST
 * hints (0 = unknown): min_m = max_m and min_n = max_n tell the planner that
 * every LP has the same size, which saves the size classification and the
 * passes of empty size classes (a wrong hint costs speed, not correctness). */
typedef struct {
  int32_t count;
  int32_t max_m, max_n;
  int32_t dtype;
  const int32_t *m, *n;
  const int64_t *a_off, *b_off, *c_off;
  const void *A, *b, *c;
  int32_t min_m, min_n;
} lpb_batch;

/* Caller-owned device outputs, FP64 whatever the input dtype.  status, iters
 * and obj have `count` entries; x is packed like c (n[k] values at c_off[k]);
 * y (the duals of A x <= b) and basis are packed like b (m[k] values at
 * b_off[k]).  basis[i] is the variable basic in row i: 0..n-1 structural,
 * n+j slack of row j, -1 for a redundant row.  Any of iters, y, basis may be
 * NULL.  For a non-optimal LP x and y are 0 and obj is -inf (infeasible),
 * +inf (unbounded) or NaN. */
typedef struct {
  int32_t *status;
  int32_t *iters;
  double *obj;
  double *x;
  double *y;
  int32_t *basis;
} lpb_result;

/* Solver options; zero-initialised fields take the defaults in brackets. */
typedef struct {
  int32_t prec;              /* lpb_precision [LPB_FP64] */
  int32_t max_iter;          /* pivot cap per LP [50 (m + n)] */
  double eps_p;              /* Step 2 eligibility t_ie > eps_p [1e-9 FP64 and the FP64 re-solve, 1e-6 FP32] */
  double eps_d;              /* Step 1 eligibility r_j < -eps_d [1e-9 FP64 and the FP64 re-solve, 1e-6 FP32] */
  double feas_tol;           /* Phase I / verification tolerance [1e-9] */
  int32_t keep_basis_inverse;/* keep what lpb_solve_backward needs in ws [0] */
  int32_t kernel;            /* lpb_kernel: force a kernel class [LPB_KERNEL_AUTO] */
  int32_t threads;           /* threads per CTA of the tableau kernel, a multiple of 32 up to 1024 [auto] */
  int32_t reg_warps;         /* warps per LP of the register kernel: 1 (m, n <= 31), 4 or 8
                                [autotuned, else 1 when every LP has m, n <= 31, else 8; with
                                kernel = AUTO and reg_warps = 0, batches of LPs with m, n <= 31
                                take the several-LPs-per-warp kernel (LPB_KERNEL_PACK), and
                                FP64-input batches (or size classes) with 32 <= max(m, n) take
                                LPB_KERNEL_WARP up to m n = 10000, and beyond that where an SM
                                holds four of its LPs (with refinement: while one register-kernel
                                CTA per SM fits)] */
  int32_t pivot_rule;        /* lpb_pivot_rule: Step 1's entering-column rule [LPB_PIVOT_LPC] */
  uint64_t seed;             /* LPB_PIVOT_RPC: seed of the counter-based random draw [0] */
} lpb_options;

/* Step 1's rule for the entering column (Section 4.2).
 *   LPB_PIVOT_LPC: "largest positive coefficient" -- the most negative reduced
 *     cost (Dantzig's rule), ties to the lowest variable index.
 *   LPB_PIVOT_RPC: "random positive coefficient" -- a uniformly random eligible
 *     column: the eligible variable j with the smallest (key, j), where the key
 *     of j at pivot t of LP k (its index in the batch) is the upper 32 bits of
 *     the first SplitMix64 output (Steele, Lea and Flood 2014) from the state
 *     seed ^ (k << 40) ^ (t << 20) ^ j.  The draw is a function of (seed, k, t,
 *     j) only, so FP64 solves repeat exactly; the FP32 register kernel ranks
 *     eligible columns by the upper 31 bits of the same key.
 *   LPB_PIVOT_STEEPEST: steepest-edge pricing (not one of the paper's rules;
 *     Goldfarb and Reid's, with exact weights read off the tableau): the
 *     eligible column j with the largest r_j^2 / gamma_j, where gamma_j = 1 +
 *     sum_i t_ij^2 over the constraint rows in use (rows left with an
 *     artificial basic variable after Phase I are not), ties to the lowest
 *     variable index.  The weights are recomputed from the tableau before
 *     every pivot: O(m n) more work per pivot for fewer pivots.  The register
 *     kernel has it in its 8-warp templates only: LPB_KERNEL_REG with
 *     reg_warps = 4 and this rule is LPB_EUNSUPPORTED.
 * Under every rule, m + n consecutive degenerate pivots switch Step 1 to the
 * lowest eligible variable index (Bland's rule) until a pivot makes progress. */
typedef enum { LPB_PIVOT_LPC = 0, LPB_PIVOT_RPC = 1, LPB_PIVOT_STEEPEST = 2 } lpb_pivot_rule;

typedef enum {
  LPB_KERNEL_AUTO = 0,
  LPB_KERNEL_SMEM = 1,   /* tableau in shared memory, one CTA per LP */
  LPB_KERNEL_GMEM = 2,   /* tableau in a per-CTA workspace slot (L2 resident) */
  LPB_KERNEL_REG = 3,    /* tableau in registers (FP32, m < 128, type 1) */
  LPB_KERNEL_PACK = 4,   /* several tiny LPs per warp: 4 (m, n <= 7), 2 (m, n <= 15) or 1
                            (m, n <= 31) register tableaux in one warp (FP32 modes,
                            largest-coefficient or random rule) */
  LPB_KERNEL_WARP = 5    /* one warp per LP, the FP32 tableau in shared memory (FP64 input,
                            m, n <= 127; FP32 modes, largest-coefficient or random rule; no
                            warm starts in lpb_solve_shared) */
} lpb_kernel;

typedef struct lpb_handle lpb_handle;

/* Create a handle bound to CUDA device `device`; allocates its counters. */
lpb_err lpb_create(lpb_handle **handle, int device);
/* Free the handle (synchronises the device first). */
lpb_err lpb_destroy(lpb_handle *handle);

/* Workspace bytes lpb_solve / lpb_solve_backward need for this batch shape
 * and these options (depends only on count, max_m, max_n, min_m, min_n,
 * dtype and the options; a solve whose batch declares other sizes than the
 * query may need more and then returns LPB_ENOMEM before any launch). */
lpb_err lpb_workspace_size(lpb_handle *handle, const lpb_batch *batch, const lpb_options *opt,
                           size_t *bytes);

/* Solve every LP of the batch (Section 3.1 Steps 1-3 with the entering rule
 * opt->pivot_rule, Dantzig's by default; Phase I of Section 3 when some
 * b_i < 0).  Asynchronous on `stream`. */
lpb_err lpb_solve(lpb_handle *handle, const lpb_batch *batch, const lpb_options *opt,
                  const lpb_result *result, void *ws, size_t ws_bytes, void *stream);

/* Vector-Jacobian product of obj and x* through the optimal basis of a
 * previous lpb_solve of the same batch with the same ws (which must have run
 * with keep_basis_inverse = 1, or the basis is refactorised).  g_obj [count]
 * and g_x (packed like c) are the upstream gradients (either may be NULL = 0).
 * Writes g_c (like c), g_b (like b), g_A (like A), all FP64 device arrays:
 *   d obj/dc = x*,  d obj/db = y,  d obj/dA = -y x*^T,
 *   for x*: v = B^{-T} g_B,  d/db += v,  d/dA += -v x*^T,  d/dc += 0.
 * Non-optimal LPs get zero gradients. */
lpb_err lpb_solve_backward(lpb_handle *handle, const lpb_batch *batch, const lpb_options *opt,
                           const lpb_result *result, const double *g_obj, const double *g_x,
                           double *g_c, double *g_b, double *g_A, void *ws, size_t ws_bytes,
                           void *stream);

/* Hyperbox support functions, Section 6 Eq. 8: for k < count,
 * obj[k] = sum_i c[k][i] * h_i with h_i = l_i if c[k][i] < 0 else u_i, summed
 * in index order from +0.0 with each product rounded (no FMA).
 * c is count x n row-major; l and u are count x n (shared_box = 0) or n values
 * (shared_box = 1); obj has count values; x (nullable) receives h, count x n.
 * All arrays have dtype `dtype` and live on the device. */
lpb_err lpb_hyperbox(lpb_handle *handle, int64_t count, int32_t n, int32_t dtype,
                     const void *c, const void *l, const void *u, int32_t shared_box,
                     void *obj, void *x, void *stream);

/* Autotuner.  Picks, for batches shaped like `batch` (same max_m, max_n,
 * dtype and precision), the fastest schedule among: warps per LP of the
 * register kernel (1, 4 or 8), the one-warp-per-LP shared-memory kernel
 * (LPB_KERNEL_WARP, where it applies), threads per CTA of the tableau kernel
 * (automatic, 256, 512 or 1024) and its placement (shared memory when it
 * fits, or L2-resident slots).
 * If `table_path` (may be NULL) holds an entry for this shape, that entry is
 * loaded and nothing is timed; otherwise every candidate solves `batch` into
 * `result` on `stream` (one warm-up and two timed runs each, CUDA events),
 * the winner is stored in the handle and appended to `table_path`.  Later
 * lpb_solve calls whose options leave kernel, threads and reg_warps at 0 use
 * the tuned schedule.  Synchronises `stream`.  *best_ms (nullable) receives
 * the winner's time per solve (0 when loaded from the table). */
lpb_err lpb_autotune(lpb_handle *handle, const lpb_batch *batch, const lpb_options *opt,
                     const lpb_result *result, void *ws, size_t ws_bytes, const char *table_path,
                     void *stream, float *best_ms);

/* Synchronise `stream`, read and clear the device error word.  Returns
 * LPB_OK or LPB_EDEVICE (word != 0; *word receives it when non-NULL). */
lpb_err lpb_sync_error(lpb_handle *handle, void *stream, uint32_t *word);

/* Counters of the last lpb_solve (synchronises `stream`): LPs re-solved in
 * FP64 after failing FP32 verification, and LPs deferred from the register
 * kernel to the shared-memory kernel. */
typedef struct {
  int64_t resolved_fp64;
  int64_t deferred;
  int64_t kernels;        /* kernel launches of the last lpb_solve on this handle */
  int64_t reserved[5];
} lpb_stats;
lpb_err lpb_get_stats(lpb_handle *handle, void *stream, lpb_stats *stats);

/* lpb_solve for a batch and results held in HOST memory: the CUDA-streams
 * pipeline of Section 4.5.  `host_batch` and `host_result` have the layout of
 * lpb_batch / lpb_result, but every pointer in them is a host pointer; the
 * offsets must increase with the LP index (each array packed in LP order, no
 * overlap; LPB_EINVAL otherwise).  The batch is cut into chunks of `chunk`
 * LPs; while chunk i is solved on `stream`, chunk i+1 is copied to the device
 * and chunk i-1's results are copied back, on two streams of the handle.  Host
 * arrays should be page-locked (cudaHostAlloc / cudaHostRegister) for the
 * copies to overlap; pageable memory works but serialises the copies with the
 * host.  `ws` is device memory of at least lpb_workspace_size_host() bytes,
 * 256-byte aligned: one solve workspace and two chunk buffer sets.  The call
 * queues the work and returns; `stream` reaches the point after the call once
 * every result is in host memory (synchronise it before reading them).  The
 * results equal those of lpb_solve on the same batch (LPB_PIVOT_RPC keys LPs
 * by their batch index).  A CUDA error after some chunks were queued returns
 * LPB_ECUDA with those chunks' work still in flight. */
lpb_err lpb_workspace_size_host(lpb_handle *handle, const lpb_batch *host_batch, const lpb_options *opt,
                                int32_t chunk, size_t *bytes);
lpb_err lpb_solve_host(lpb_handle *handle, const lpb_batch *host_batch, const lpb_options *opt,
                       const lpb_result *host_result, int32_t chunk, void *ws, size_t ws_bytes, void *stream);

/* Shared-constraint batches: the support function of one polytope in many
 * directions, Section 6's application (sampling the support function of
 * {A x <= b, x >= 0} along `count` directions).  For k < count:
 *
 *     maximize  C[k]^T x   subject to  A x <= b,  x >= 0,
 *
 * with one A (m x n row-major) and b (m) shared by every LP, C count x n
 * row-major; A, b and C have dtype `dtype` and live on the device.  Results
 * (device, caller-owned, FP64): status, iters, obj per direction; x of LP k at
 * k n (count x n); y and basis (nullable) of LP k at k m (count x m).  Every
 * LP reads the one copy of A and b, which stays in L2 across the batch; the
 * solve is otherwise that of lpb_solve (all precisions, pivot rules, Phase I
 * when some b_i < 0).  `ws` is device memory of lpb_workspace_size_shared()
 * bytes, 256-byte aligned.  Asynchronous on `stream`. */
lpb_err lpb_workspace_size_shared(lpb_handle *handle, int32_t m, int32_t n, int32_t dtype, int64_t count,
                                  const lpb_options *opt, size_t *bytes);
lpb_err lpb_solve_shared(lpb_handle *handle, int32_t m, int32_t n, int32_t dtype, const void *A, const void *b,
                         int64_t count, const void *C, const lpb_options *opt, const lpb_result *result,
                         void *ws, size_t ws_bytes, void *stream);

/* Bounded variables: for every LP of the batch
 *
 *     maximize  c^T x   subject to  A x <= b,  l <= x <= u,
 *
 * with l and u (device, FP64, packed like c) in place of x >= 0; l must be
 * finite, u may be +inf.  Solved exactly through the change of variables
 * x = l + z: max c^T z + c^T l subject to A z <= b - A l (formed in FP64),
 * z_j <= u_j - l_j (the row 0 <= 1 when u_j = +inf) and z >= 0 -- an LP of
 * m + n rows that lpb_solve's passes handle (all precisions and pivot rules;
 * an empty box or b - A l < 0 goes through Phase I).  The batch must be FP64
 * (LPB_EUNSUPPORTED otherwise).  Results: status, iters, obj and x of the
 * bounded LP (x = l + z), y the duals of A x <= b (nullable); result->basis
 * must be NULL (LPB_EINVAL), the basis of the reduced LP having m + n rows.
 * `ws` is device memory of lpb_workspace_size_bounded() bytes (the reduced
 * batch at a fixed stride of (max_m + max_n) x max_n per LP, plus a solve
 * workspace), 256-byte aligned.  Asynchronous on `stream`. */
lpb_err lpb_workspace_size_bounded(lpb_handle *handle, const lpb_batch *batch, const lpb_options *opt,
                                   size_t *bytes);
lpb_err lpb_solve_bounded(lpb_handle *handle, const lpb_batch *batch, const void *l, const void *u,
                          const lpb_options *opt, const lpb_result *result, void *ws, size_t ws_bytes,
                          void *stream);

/* lpb_solve for callers that cannot allocate device memory.  The paper has no
 * counterpart; this exists for plug-ins whose host framework owns all device
 * memory through its own pool, and for loops where cudaMalloc / cudaFree are
 * not allowed because they can synchronise the device.
 *
 * Same arguments and results as lpb_solve, minus the handle and workspace: it
 * solves on the current CUDA device and takes its scratch from a 32 MiB
 * device array inside the library (every GPU on which the library's module
 * is loaded holds that array until the process exits).  It allocates nothing:
 * no cudaMalloc, cudaFree or allocating library call.
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Returns LPB_ENOMEM, before launching anything, when the batch needs more
 *     scratch than the array holds (lpb_workspace_size gives the need).
 *   - Every call on a device shares the one array and starts by clearing its
 *     counters and error word; calls that overlap on the GPU race on it, so
 *     run them one after another. */
lpb_err lpb_solve_noalloc(const lpb_batch *batch, const lpb_options *opt, const lpb_result *result,
                          void *stream);

/* The device error word of lpb_solve_noalloc, which lives in the same fixed
 * array (the paper has no counterpart; see lpb_solve_noalloc).  Synchronises
 * `stream`, copies the word of the current device into *word (when non-NULL)
 * and clears it.  Returns LPB_OK (word == 0), LPB_EDEVICE (a kernel of an
 * earlier lpb_solve_noalloc recorded a fault: the bits are those that
 * lpb_sync_error reports) or LPB_ECUDA.  Read it before the next
 * lpb_solve_noalloc on the device, which starts by clearing the word.
 * Allocates nothing. */
lpb_err lpb_noalloc_sync_error(void *stream, uint32_t *word);

/* Kernel timing.  lpb_profile_start(h, calls) makes the next `calls` (<= 256)
 * lpb_solve calls record a CUDA event pair on their stream around each of
 * their kernel passes (pass 0: every LP; pass 1: LPs needing more artificial
 * columns; pass 2: the FP64 re-solve).  lpb_profile_read synchronises those
 * events, writes ms[3 * i + p] = milliseconds of pass p in recorded call i
 * (0 when the pass did not launch), sets *ncalls and stops recording. */
lpb_err lpb_profile_start(lpb_handle *handle, int32_t calls);
lpb_err lpb_profile_read(lpb_handle *handle, float *ms, int32_t max_calls, int32_t *ncalls);

const char *lpb_strerror(lpb_err err);
const char *lpb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LPB_H_ */
