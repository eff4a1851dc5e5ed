/*
 * lqt.h -- C ABI of the GB300 (sm_103a) temporally parallel LQT solver.
 *
 * The library solves the linear quadratic tracking (LQT) problem of
 * Särkkä & García-Fernández, "Temporal Parallelisation of Dynamic Programming
 * and Linear Quadratic Control", Sec. II-B, eq. LQT_problem:
 *
 *     x_{k+1} = F_k x_k + c_k + L_k u_k,                       k = 0..T-1
 *     cost    = 1/2 (H_T x_T - r_T)^T X_T (H_T x_T - r_T)
 *             + sum_k 1/2 (H_k x_k - r_k)^T X_k (H_k x_k - r_k) + 1/2 u_k^T U_k u_k
 *
 * with X_k, X_T symmetric positive semi-definite and U_k symmetric positive
 * definite, and returns the value function V_k(x) = z + 1/2 x^T S_k x - v_k^T x
 * (eq. V_k_LQT), the feedback gains K_k of the control law eq. Control_LQT, the
 * optimal states x*_k and the optimal controls u*_k.
 *
 * Method (Sec. IV and V-A): per-step elements (A, b, C, eta, J) of eq. lqt_init,
 * a backward parallel scan with the associative operator of eq. lqt_comb
 * (Lemma LQT_combination) giving S_k = J_{k,T+1} and v_k = eta_{k,T+1}
 * (Lemma LQT_assoc), and a forward parallel scan of the closed-loop affine maps
 * (Lemma LQT_trajectory_combination, Lemma lqt_fwd_init: "Method 1").
 * Scans are blocked (Sec. V-C): sequential folds over chunks of steps, and
 * up/down sweeps (Sec. II-C, Alg. 1) over the chunk totals.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major, per-step arrays are time-major and densely packed
 *     within one step.  A step stride (in elements) of 0 means the same matrix
 *     at every step.
 *   - dtype LQT_F32 means every input and output is float, LQT_F64 double.
 *   - Unless an entry point says otherwise, every pointer is a DEVICE pointer
 *     owned by the caller; inputs are only read.  The library allocates no
 *     device memory: scratch space is the caller's workspace.
 *   - Every pointer must be aligned to its element size; workspace pointers to
 *     256 bytes.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Solves are asynchronous: the return value reports argument
 *     validation and launch errors only.  Numerical failures found on the
 *     device are reported by lqt_workspace_status().
 *   - Entry points are thread-safe except lqt_profile_enable/lqt_profile_read,
 *     which keep process-wide state.
 */
#ifndef LQT_H
#define LQT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LQT_OK = 0,
    LQT_EINVAL = 1,       /* invalid argument (sizes, NULL pointer, alignment) */
    LQT_ENOTSPD = 2,      /* L^T S L + U or U was not positive definite at some step */
    LQT_ENONFINITE = 3,   /* a non-finite value appeared in the outputs */
    LQT_ENOMEM = 4,       /* the workspace passed in is smaller than required */
    LQT_ECUDA = 5,        /* a CUDA runtime call failed */
    LQT_ETIMEOUT = 6,     /* a bounded device wait ran out */
    LQT_EUNSUPPORTED = 7, /* no kernel compiled for this (n, m, dtype) */
    LQT_ESINGULAR = 8     /* I + C J was numerically singular in a combine */
} lqt_status;

typedef enum { LQT_F32 = 0, LQT_F64 = 1 } lqt_dtype;

/* One per-step input: base pointer and the distance between consecutive steps
 * in elements (0 = time-invariant). */
typedef struct {
    const void *ptr;
    int64_t step_stride;
} lqt_in;

/* The problem of eq. LQT_problem with S = 0 (Sec. II-A numbering k = 0..T).
 *   n = state size nx, m = control size nu, p = rows of H_k, pT = rows of H_T.
 *   F : n x n,  c : n (ptr may be NULL: c_k = 0),  L : n x m,  U : m x m
 *   H : p x n,  r : p (ptr may be NULL: r_k = 0),  X : p x p        (k = 0..T-1)
 *   HT: pT x n, rT: pT (may be NULL), XT: pT x pT                   (terminal)
 *   x0: n                                                             (initial state)
 * The stride of a time-varying input must be at least its per-step size. */
typedef struct {
    int32_t n, m, p, pT;
    int64_t T;
    int32_t dtype; /* lqt_dtype */
    lqt_in F, c, L, U;
    lqt_in H, r, X;
    const void *HT, *rT, *XT;
    const void *x0;
} lqt_problem;

/* Outputs (caller-allocated, contiguous, dtype of the problem):
 *   S: (T+1) x n x n   value-function matrices S_0..S_T   (eq. V_k_LQT)
 *   v: (T+1) x n       value-function vectors  v_0..v_T
 *   K: T x m x n       feedback gains K_0..K_{T-1}        (eq. Control_LQT)
 *   x: (T+1) x n       optimal states x*_0..x*_T          (x*_0 = x0)
 *   u: T x m           optimal controls u*_0..u*_{T-1}
 * Output arrays must not overlap each other or any input. */
typedef struct {
    void *S, *v, *K, *x, *u;
} lqt_solution;

/* Solver options.  Pass NULL for the defaults (refine = LQT_REFINE_AUTO).
 *
 * refine: mixed-precision iterative refinement.  The optimal control
 *   u*_k = -K_k x*_k + d_k is often a small difference of large terms
 *   (tracking a slowly varying reference), so FP32 rounding of S, v and x is
 *   amplified in u*; ill-conditioned costs amplify it in every output.
 *   n <= 4 (LQT_REFINE_ON and LQT_REFINE_FULL alike): the solve runs twice,
 *   first on the problem, then on the same problem shifted by the first
 *   trajectory x^ (x = x^ + xi: r'_k = r_k - H_k x^_k,
 *   c'_k = F_k x^_k + c_k - x^_{k+1}, r'_T = r_T - H_T x^_T, x'_0 = 0), whose
 *   residual terms are formed with compensated (twice-working-precision) dot
 *   products; it returns u* directly and x* = x^ + xi.  S, v, K come from
 *   the first solve.
 *   n = 8, 16, 32 (FP32 problems): LQT_REFINE_ON takes one step of iterative
 *   refinement of the KKT system of the QP: the residuals of the dynamics and
 *   of the optimality
 *   conditions in x and u at the first solve (x^, u^, lambda^_k =
 *   S_k x^_k - v_k) are formed in FP64, a second solve of the correction
 *   problem (same matrices, linear state terms, offsets) gives (dx, du), and
 *   x* = x^ + dx, u* = u^ + du.  LQT_REFINE_FULL also runs the tree levels
 *   above the chunks in FP64 and takes one Newton step of the Riccati
 *   recursion for S, v and K: the residuals
 *   R_k = Ric_k(S^_{k+1}) - S^_k are formed in FP64, the linear recursion
 *   dS_k = Phi_k^T dS_{k+1} Phi_k + R_k (closed loop Phi_k) is solved by the
 *   same scan, and K_k is recomputed in FP64 from S^ + dS.  FP64 arithmetic is
 *   slow on this GPU, so FULL costs several times ON.
 *   LQT_REFINE_AUTO = LQT_REFINE_ON for FP32 solves, OFF for FP64 ones. */
enum { LQT_REFINE_OFF = 0, LQT_REFINE_ON = 1, LQT_REFINE_AUTO = 2, LQT_REFINE_FULL = 3 };
/* method: trajectory recovery (Sec. IV-C).  LQT_METHOD_DEFAULT (0) and
 *   LQT_METHOD_1 take Method 1 (Lemma LQT_trajectory_combination: a forward
 *   scan of the closed-loop affine maps from x_0).  LQT_METHOD_2 (n = 8, 16, 32
 *   only; LQT_EUNSUPPORTED otherwise) takes Method 2 (Lemma
 *   LQT_trajectory_method2): a forward scan of the same elements seeded with
 *   (0, x_0, 0, 0, 0) (Remark LQT_init2) gives V_{S->k}, and
 *   x*_k = (I + C_{S,k} S_k)^{-1} (b_{S,k} + C_{S,k} v_k) (eq. lqt_method_2);
 *   u*_k follows from the control law. */
enum { LQT_METHOD_DEFAULT = 0, LQT_METHOD_1 = 1, LQT_METHOD_2 = 2 };
/* wait_probe_polls: diagnostic of the bounded device waits (n <= 4 sizes
 *   only; LQT_EUNSUPPORTED elsewhere).  0 (the default) does nothing.  When
 *   positive, the backward down-sweep kernel of each pass also waits on a
 *   barrier that nothing completes, giving up after this many polls: exactly
 *   what a bulk copy that never lands would cause.  The wait runs out, the
 *   kernel records LQT_ETIMEOUT in the status word and carries on, so the
 *   solve still writes its outputs and lqt_workspace_status() returns
 *   LQT_ETIMEOUT.  No copy is attached to that barrier, so nothing is left in
 *   flight.  The real bulk copies always wait with the library's own limit
 *   (2^24 polls).  Used by the tests of the timeout path. */
typedef struct {
    int32_t refine;
    int32_t method;
    int32_t wait_probe_polls;
    int32_t reserved[5]; /* must be 0 */
} lqt_options;

/* Bytes of device workspace that lqt_solve needs for this problem and these
 * options (0 on invalid arguments or an unsupported size).  Depends on n, m,
 * p, pT, T, dtype, the options and the current device's SM count. */
size_t lqt_workspace_bytes(const lqt_problem *prob, const lqt_options *opts);

/* Temporally parallel LQT solve (Sec. V-A: initialisation, backward scan and
 * extraction, then the Method-1 forward scan), asynchronous on `stream`.
 * `workspace` is a device buffer of at least lqt_workspace_bytes(prob) bytes,
 * 256-byte aligned, used by this call until the stream reaches the end of the
 * solve; its first bytes hold the device status word read by
 * lqt_workspace_status().  Between its kernels the solve keeps the
 * feedforward terms of the control law in the u output.
 * Returns LQT_EINVAL / LQT_ENOMEM / LQT_EUNSUPPORTED / LQT_ECUDA on failure,
 * before or while launching; nothing is written in the first three cases. */
lqt_status lqt_solve(const lqt_problem *prob, const lqt_solution *sol, const lqt_options *opts,
                     void *workspace, size_t workspace_bytes, void *stream);

/* Single-tile solves (n <= 4 thread-per-chunk path; a property of this
 * implementation, not of the paper).  Each thread of a tile folds a chunk of
 * consecutive steps (Sec. V-C block processing) and a tile's W chunks are
 * scanned in shared memory (Alg. 1).  A problem with 0 < T <= W x
 * max_chunk_steps (W = 512 threads in FP32, 256 in FP64) runs in a single CTA:
 * each pass (two when refining) is one launch that keeps the in-tile trees in
 * shared memory, where a longer problem takes five launches per pass over
 * many tiles.  0 turns single-tile solves off.  Default 2 (T <= 1024 in
 * FP32).  The setting is process-wide; solves already launched are not
 * affected.  *previous (may be NULL) receives the old value.  Returns
 * LQT_EINVAL for a negative value. */
lqt_status lqt_set_single_tile_chunk(int32_t max_chunk_steps, int32_t *previous);

/* Sequential Riccati recursion of Sec. II-B followed by the forward pass of
 * eq. optimal_trajectory, run on the GPU by one thread per problem (the
 * sequential baseline).  Same problem, options, outputs and workspace rules
 * as lqt_solve (lqt_workspace_bytes with the same options suffices). */
lqt_status lqt_riccati_sequential(const lqt_problem *prob, const lqt_solution *sol,
                                  const lqt_options *opts, void *workspace,
                                  size_t workspace_bytes, void *stream);

/* Synchronises `stream` and returns the device status word of the last solve
 * that used `workspace`: LQT_OK, LQT_ENOTSPD, LQT_ENONFINITE, LQT_ESINGULAR or
 * LQT_ETIMEOUT (a bounded device wait ran out; the outputs are then not to be
 * trusted), or LQT_ECUDA if the read itself failed.  The next solve on the
 * workspace clears the word first. */
lqt_status lqt_workspace_status(const void *workspace, void *stream);

/* Host-buffer solve: every pointer in `host_prob` and `host_sol` is a HOST
 * pointer (pinned memory gives full copy speed).  The inputs are copied into
 * `device_buffer` (a device buffer of at least lqt_host_solve_bytes(host_prob,
 * opts) bytes, 256-byte aligned), lqt_solve runs there, and the outputs are copied
 * back; the call synchronises `stream` and returns the device status of the
 * solve.  At the thread-per-chunk sizes (n <= 4) S, v and K are copied back on
 * an internal stream as soon as the first pass's backward scan has written
 * them, while the rest of the solve runs.  That stream and two events are
 * created on a host thread's first call for a device and are kept until the
 * process exits (they are not released when the thread ends).
 * Several host threads may call it at once, each with its own stream, device
 * buffer and host buffers; one caller's copies then overlap another's
 * kernels.  Returns LQT_EINVAL, LQT_ENOMEM, LQT_EUNSUPPORTED or LQT_ECUDA on
 * failure. */
size_t lqt_host_solve_bytes(const lqt_problem *host_prob, const lqt_options *opts);
lqt_status lqt_solve_host(const lqt_problem *host_prob, const lqt_solution *host_sol,
                          const lqt_options *opts, void *device_buffer, size_t device_bytes,
                          void *stream);

/* Ragged batch of independent problems (any mix of T and of the compiled
 * batch sizes (n, m) in {(4,2), (8,4), (16,8), (32,16)}; FP32; p, pT <= 2n),
 * each solved by the temporally parallel method of lqt_solve (Sec. V-A,
 * Method 1; chunked as in Sec. V-C):
 *   n = 4:  one persistent launch; each problem runs inside one CTA, its steps
 *           cut into chunks (one group of 4 lanes per chunk) whose totals are
 *           swept in shared memory (Alg. 1); CTAs take problems from a work
 *           queue.
 *   n >= 8: the chunked pipeline of lqt_solve with all problems of one size
 *           in each of its launches: every problem's steps are cut into a
 *           power-of-two number of chunks (of the length lqt_batch_set_tuning
 *           sets, by default at most 64 steps), whose results are swept tree
 *           level by tree level, by one launch per level or by one
 *           cooperative launch per size (the launch mode of
 *           lqt_batch_set_tuning).
 *   items: HOST array of `count` descriptors; each holds device pointers to a
 *          problem's inputs and outputs, with the layouts of lqt_problem and
 *          lqt_solution.  The array may be reused when the call returns.
 *   workspace: device buffer of at least lqt_batch_workspace_bytes(items,
 *          count) bytes (0 means an invalid or unsupported item), 256-byte
 *          aligned; its first bytes hold the status word read by
 *          lqt_workspace_status().  The size depends on the problems' n and T.
 * No refinement is applied (problems whose controls cancel, see lqt_options,
 * should use lqt_solve).  Asynchronous on `stream`: the descriptors built from
 * `items` reach the workspace as kernel parameters, so the call never waits
 * for the stream, and it may be captured in a CUDA graph (the graph keeps the
 * descriptors; replays solve the same problems, reading whatever their input
 * buffers hold then).  A batch of at least 2^20 steps in all runs its lane
 * sizes side by side on streams of the calling host thread (created on its
 * first such call on a device and kept until the process exits: make that
 * first call before any stream capture), forked from and joined back to
 * `stream` with events; the outputs are those of one stream, bit for bit.
 * Returns LQT_EINVAL, LQT_EUNSUPPORTED, LQT_ENOMEM or LQT_ECUDA on argument or
 * launch errors.  Work queued before a launch error stays queued, ordered
 * before whatever the caller queues next on `stream` (the side streams are
 * joined back on every return): keep the workspace and outputs until
 * `stream` has passed that point. */
typedef struct {
    lqt_problem problem;
    lqt_solution solution;
} lqt_batch_item;

size_t lqt_batch_workspace_bytes(const lqt_batch_item *items, int32_t count);
lqt_status lqt_solve_batched(const lqt_batch_item *items, int32_t count, void *workspace,
                             size_t workspace_bytes, void *stream);

/* Launch plan of lqt_solve_batched for the lane-group sizes (n >= 8; not in
 * the paper: a property of this implementation).  Each problem's steps are
 * cut into a power-of-two number of chunks, one lane group per chunk (Sec. V-C
 * block processing); by default the chunk length is the batch's total steps
 * over the resident lane groups, clamped to [4, 64].  An entry {n, t_max,
 * chunk_steps} sets the chunk length of the problems of state size n with
 * T <= t_max (the first matching entry applies), capped at the batch's total
 * steps over the resident lane groups (at least 4), so that a batch too small
 * to fill the device with chunks of that length still spreads over every
 * resident group; `persistent` selects the launch mode: one launch per tree
 * level (LQT_BATCH_PER_LEVEL), one cooperative launch per state size that
 * runs every tree level with grid barriers (LQT_BATCH_PERSISTENT), or
 * (LQT_BATCH_AUTO, the default) the cooperative launch when its grid (one lane
 * group per chunk) needs at most half of the CTAs the device holds at once,
 * per-level launches otherwise.  The persistent launch saves the launch gaps
 * that dominate small batches; a larger cooperative launch waits until its
 * whole grid is resident, which serialises it with the work of other
 * streams, and with many waves of chunks the per-level kernels, whose blocks
 * are sized per phase, keep more groups busy.  count = 0
 * clears the table.  The settings are process-wide; calls already launched
 * are not affected.  Returns LQT_EINVAL for more than 64 entries, a
 * non-positive n or chunk length, or another launch mode.  The Python binding
 * applies the table that paper_2104_03186_gb300/tune.py measured on this GPU
 * model. */
enum { LQT_BATCH_PER_LEVEL = 0, LQT_BATCH_PERSISTENT = 1, LQT_BATCH_AUTO = 2 };
typedef struct {
    int32_t n;
    int32_t chunk_steps;
    int64_t t_max;
} lqt_batch_tune_entry;
lqt_status lqt_batch_set_tuning(const lqt_batch_tune_entry *entries, int32_t count,
                                int32_t persistent);

/* Warm solves: problems whose S_k and K_k are already known.
 *
 * S_k and K_k depend on the matrices F, L, U, H, X and the terminal H_T, X_T
 * only: the Riccati recursion of Sec. II-B never reads r, c or x_0.  A
 * problem over steps [s, s + T) of a model that an earlier solve covered over
 * [0, s + T) with the same terminal weights (a receding horizon, as in model
 * predictive control) therefore has S_k = S'_{s+k} and K_k = K'_{s+k} of the
 * earlier solve, whatever its own references, offsets and initial state.
 * This call takes them as given and computes the rest by the vector
 * recursions of Sec. II-B with the closed loop Ft_k = F_k - L_k K_k:
 *   v_T = H_T^T X_T r_T,  v_k = Ft_k^T (v_{k+1} - S_{k+1} c_k) + H_k^T X_k r_k,
 *   d_k = (L_k^T S_{k+1} L_k + U_k)^{-1} L_k^T (v_{k+1} - S_{k+1} c_k),
 *   u*_k = -K_k x*_k + d_k,  x*_{k+1} = F_k x*_k + c_k + L_k u*_k,
 * each scanned over chunks of steps as an affine recursion (Sec. IV-C),
 * which costs one n x n product and one m x m solve per step instead of the
 * full solve's element folds and Riccati steps.
 *   items: HOST array of `count` problems (any mix of dtype FP32 / FP64 and
 *          of the sizes (n, m) in {(4,2), (8,4), (16,8), (32,16)}; p, pT <=
 *          2n), with the layouts of lqt_problem and lqt_solution.  On entry
 *          solution.S ((T+1) x n x n) and solution.K (T x m x n) must hold
 *          the known S_k and K_k; they are read, never written, so they may
 *          point into an earlier solve's outputs at step offset s.  v, x, u
 *          are written.  The array may be reused when the call returns.
 *   workspace: device buffer of at least lqt_warm_workspace_bytes(items,
 *          count) bytes (0: an invalid or unsupported item), 256-byte
 *          aligned; its first word is the status word of
 *          lqt_workspace_status() (LQT_ENOTSPD when some
 *          L_k^T S_{k+1} L_k + U_k is not positive definite).
 * Asynchronous on `stream`; returns LQT_EINVAL, LQT_EUNSUPPORTED, LQT_ENOMEM
 * or LQT_ECUDA on argument or launch errors.  The result equals that of a
 * full solve of the same problem up to rounding when the given S and K are
 * that problem's. */
size_t lqt_warm_workspace_bytes(const lqt_batch_item *items, int32_t count);
lqt_status lqt_solve_warm(const lqt_batch_item *items, int32_t count, void *workspace,
                          size_t workspace_bytes, void *stream);

/* Solve without any caller-provided workspace.
 *
 * There is no counterpart to this entry point in the paper.  It exists for
 * callers that cannot allocate device memory for a workspace: for example a
 * real-time control loop that forbids allocation once it has started, or a
 * host framework that owns the device allocator and has no way to hand this
 * library a buffer.  It runs exactly lqt_solve, but its scratch space is one
 * fixed array of LQT_STATIC_SCRATCH_BYTES compiled into the library: every GPU
 * that loads the library holds that array until the process exits.
 *
 *   - Inputs and outputs are still the caller's device buffers, as for
 *     lqt_solve.  Nothing is allocated: no cudaMalloc, no cudaFree.
 *   - Problems whose lqt_workspace_bytes(prob, opts) exceeds
 *     LQT_STATIC_SCRATCH_BYTES are rejected with LQT_ENOMEM before anything is
 *     launched.  At n = 4, p = 2 on a 152-SM GPU that is T above about 4e5
 *     with refinement; without refinement the need stays near 20 MB for any T
 *     (the launch plan keeps about one tile per SM).
 *   - The first call on a device looks up the array's device address for that
 *     device (the device must be current) and keeps it for later calls.  Make
 *     that first call before any stream capture.  A failed look-up returns
 *     LQT_ECUDA.  The kept address belongs to the device's current context:
 *     after cudaDeviceReset the library's module is loaded again and the array
 *     may move, so do not call this entry point after a device reset.
 *   - All calls share the one array, and it keeps the last call's contents.
 *     Calls whose work overlaps on the GPU (different streams, or several host
 *     threads) race on it and give wrong results: serialise them.
 *   - The call waits for `stream` to finish the solve (a stream
 *     synchronisation, so the call itself cannot be recorded into a CUDA
 *     graph) and returns the device status of that solve (LQT_OK,
 *     LQT_ENOTSPD, LQT_ENONFINITE or LQT_ESINGULAR), or the argument and
 *     launch errors of lqt_solve. */
#define LQT_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
lqt_status lqt_solve_static(const lqt_problem *prob, const lqt_solution *sol,
                            const lqt_options *opts, void *stream);

/* Generalised stage cost (Sec. IV-D, eq. generalised_cost): the stage cost of
 * eq. LQT_problem becomes
 *     1/2 e_k^T X_k e_k + e_k^T M_k (u_k - s_k) + 1/2 (u_k - s_k)^T U_k (u_k - s_k),
 *     e_k = H_k x_k - r_k,
 * with a cross weight M_k (p x m, row-major) and a control offset s_k (m);
 * the joint weight [[X_k, M_k], [M_k^T, U_k]] must be positive semi-definite
 * with U_k positive definite.  The terminal cost is unchanged.
 *   M, s: per-step inputs as in lqt_problem (ptr NULL: zero; step stride 0:
 *         time-invariant), device pointers, dtype of the problem.
 * A NULL `cross` means M = 0, s = 0. */
typedef struct {
    lqt_in M;
    lqt_in s;
} lqt_cross;

/* Bytes of device workspace lqt_solve_cross needs (0 on invalid arguments or
 * an unsupported size): the workspace of lqt_solve for the problem plus the
 * transformed per-step matrices. */
size_t lqt_cross_workspace_bytes(const lqt_problem *prob, const lqt_cross *cross,
                                 const lqt_options *opts);

/* Solves the generalised-cost problem by the paper's reduction to
 * eq. LQT_problem (Sec. IV-D): with W_k = U_k^{-1} M_k^T, a transform kernel
 * writes F~_k = F_k - L_k W_k H_k, c~_k = c_k + L_k (W_k r_k + s_k) and
 * X~_k = X_k - M_k W_k into the workspace (time-invariant where all their
 * inputs are), lqt_solve solves the transformed problem (same options, so
 * refinement and Method 2 apply to it), and a post kernel returns the outputs
 * of the original problem: S_k, v_k and x*_k as solved, the gain of the
 * original control law K_k = K~_k + W_k H_k, and
 * u*_k = u~*_k - W_k (H_k x*_k - r_k) + s_k.  The transform runs in the
 * problem's dtype.  Workspace rules, outputs and return values are those of
 * lqt_solve; a U_k that is not positive definite is reported as LQT_ENOTSPD
 * by lqt_workspace_status. */
lqt_status lqt_solve_cross(const lqt_problem *prob, const lqt_cross *cross,
                           const lqt_solution *sol, const lqt_options *opts, void *workspace,
                           size_t workspace_bytes, void *stream);

/* Iterated nonlinear LQT (Sec. IV-D, "Extension to nonlinear control"):
 * dynamics x_{k+1} = f(x_k, u_k) of a built-in model, the quadratic tracking
 * cost of lqt_problem (H, r, X, U and the terminal terms; h(x) = H x,
 * g(u) = u).  Each pass linearises f around the nominal trajectory by its
 * first-order Taylor series (eq. nonlinear_linarisation), solves that LQT
 * problem with lqt_solve (or the sequential recursion), and takes the optimal
 * trajectory as the next nominal.  The first nominal is x_init (or x_0 at
 * every step) and u_init (or 0).
 *   LQT_MODEL_UNICYCLE (Sec. VI-E; n = 4, m = 2): state (p_x, p_y, theta, s),
 *   control (a, omega), f = (p_x + s cos(theta) dt, p_y + s sin(theta) dt,
 *   theta + omega dt, s + a dt). */
enum { LQT_MODEL_UNICYCLE = 1 };
typedef struct {
    int32_t model;        /* LQT_MODEL_* */
    int32_t iterations;   /* linearise-and-solve passes, at least 1 */
    int32_t sequential;   /* 0: lqt_solve per pass; 1: lqt_riccati_sequential */
    int32_t reserved;     /* must be 0 */
    double dt;            /* time step of the model */
    const void *x_init;   /* (T+1) x n device array of the problem's dtype, or NULL */
    const void *u_init;   /* T x m device array, or NULL */
} lqt_nonlinear;

/* Bytes of device workspace lqt_solve_nonlinear needs (0 on invalid
 * arguments or an unsupported size). */
size_t lqt_nonlinear_workspace_bytes(const lqt_problem *prob, const lqt_nonlinear *nl,
                                     const lqt_options *opts);

/* Runs nl->iterations passes on `stream` (asynchronous).  prob supplies n, m,
 * p, pT, T, dtype, the cost (H, r, X, U, HT, rT, XT) and x_0; its F, c and L
 * are ignored.  Each pass solves the linearised problem in state deviations
 * from the nominal (same minimiser, offsets that stay small) with `opts`;
 * the nominal itself is kept in FP64 for either dtype.
 * Outputs: S_k, K_k and v_k (absolute coordinates) of the last linearisation,
 * and x*, u* of the last pass (the final nominal).  Workspace rules and return
 * values are those of lqt_solve; the device status is read with
 * lqt_workspace_status. */
lqt_status lqt_solve_nonlinear(const lqt_problem *prob, const lqt_nonlinear *nl,
                               const lqt_solution *sol, const lqt_options *opts, void *workspace,
                               size_t workspace_bytes, void *stream);

/* Partial condensing (Sec. V-C, "Block processing"): the problem is rewritten
 * in blocks of B steps whose state is the block's first state and whose
 * control is the stack of the block's B controls.  Eliminating the states
 * inside each block gives an LQT problem of ceil(T / B) steps with n states,
 * B m controls and the generalised stage cost of Sec. IV-D (the block's
 * intermediate tracking costs couple its first state and its controls), which
 * lqt_solve_cross solves.  An expansion kernel then re-runs each block's B
 * Riccati steps and its rollout, so `sol` receives S, v, K, x*, u* at every
 * step, as from lqt_solve (a shorter last block is padded with steps that
 * change nothing).  Where the condensed size (n, B m) is compiled -- FP32
 * (n, m, B) in {(2,1,2), (3,1,2), (4,1,2), (4,1,4), (4,2,2)}, FP64 (4,1,2),
 * with p <= 8 -- the condensed problem is solved as it stands.  Otherwise, for
 * FP32 (n, m) in {(4,2), (4,1), (2,1), (2,2), (1,1)} with B m <= 32 and
 * B p <= 32, each block is reduced exactly to n controls: the controls reach
 * the next block only through w = L_bar u_bar (n values), the best stacked
 * control for given block start and w is eliminated in FP64, and the reduced
 * problem (n states, n controls, B p outputs, generalised cost) is solved at
 * (n, n); the stacked controls are rebuilt from its solution before the
 * expansion.  A block that cannot move the state in every direction (a last
 * block of fewer than n / m steps) keeps the directions it can.  B = 1 is
 * lqt_solve itself.  Refinement (opts->refine; AUTO = ON for FP32): the
 * expansion rebuilds u from block starts and references of order one, so
 * with LQT_REFINE_ON or FULL the whole condensed solve runs twice, the second
 * time on the problem shifted by the first trajectory x^ (the shift of
 * lqt_options.refine for n <= 4, formed in compensated arithmetic), whose
 * controls are u* and whose states are added to x^; S, v, K are the first
 * solve's.  The condensed problem itself is solved without refinement.
 * Workspace and return values as for lqt_solve (LQT_EUNSUPPORTED for other
 * sizes and for T = 0). */
size_t lqt_condensed_workspace_bytes(const lqt_problem *prob, int32_t B, const lqt_options *opts);
lqt_status lqt_solve_condensed(const lqt_problem *prob, int32_t B, const lqt_solution *sol,
                               const lqt_options *opts, void *workspace, size_t workspace_bytes,
                               void *stream);

/* Static string for a status code (never NULL). */
const char *lqt_strerror(lqt_status status);

/* Per-kernel timing of lqt_solve.  While enabled, each lqt_solve records CUDA
 * events on its stream around every kernel it launches.  lqt_profile_read
 * waits for the last profiled solve and fills up to `max_entries` durations
 * (milliseconds) and static kernel names; it returns the number of kernels of
 * that solve (0 if none was profiled, -1 on a CUDA error).  Process-wide state:
 * not for concurrent use from several threads. */
lqt_status lqt_profile_enable(int enable);
int lqt_profile_read(float *ms, const char **names, int max_entries);

/* Launch geometry lqt_solve would use: steps per chunk, threads per tile,
 * number of tiles, kernels launched per solve (with these options).
 * Returns LQT_EINVAL / LQT_EUNSUPPORTED / LQT_ECUDA. */
lqt_status lqt_plan(const lqt_problem *prob, const lqt_options *opts, int32_t *chunk_steps,
                    int32_t *tile_threads, int32_t *tiles, int32_t *kernels);

#ifdef __cplusplus
}
#endif

#endif /* LQT_H */
