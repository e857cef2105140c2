/*
 * wlr.h -- C ABI of the GB300 sWLR library (libwlr.so).
 *
 * Solves the special weighted low-rank approximation of Dutta & Li,
 * "A Fast Algorithm for a Weighted Low Rank Approximation" (arXiv 1703.06303):
 *
 *     min_{X1, X2 : rank(X1 X2) <= r}  ||(A1 - X1) o W1||_F^2 + ||A2 - X2||_F^2     (Eq. 5)
 *
 * with A = (A1 A2) in R^{m x n}, A1 the first k columns (the weighted frames), and
 * W1 in R^{m x k}, W1 > 0 (Theorem 2 needs strictly positive weights).  The solver is
 * Algorithm 1 (sWLR): per iteration p
 *     X1_p = Q_p R_p,  C_p = R_p^{-1} Q_p^T A2,  D_p = H_{r-k}((I - Q_p Q_p^T) A2),
 *     E_p = A1 o W1 o W1 + (A2 - D_p) C_p^T,
 *     X1_{p+1}(i,:) = E_p(i,:) (diag(W1(i,:)^2) + C_p C_p^T)^{-1}   for every row i.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major with a leading dimension (columns = video frames,
 *     rows = pixels).  A is m x n with lda >= m; W1 and X1 are m x k.
 *   - Pointers are plain host or device pointers; the memory argument says which.
 *     Caller-owned device buffers passed to wlr_set_data are borrowed (not copied,
 *     not modified) when their dtype matches the handle's precision and they are
 *     device memory; they must then stay valid until wlr_destroy or the next
 *     wlr_set_data.  In every other case the library copies them.
 *   - The library owns all of its workspace; it allocates in wlr_create and frees in
 *     wlr_destroy.
 *   - Work is issued on the handle's CUDA stream.  Entry points that return a host
 *     scalar or copy into host memory synchronise that stream; the others are
 *     asynchronous.
 *   - Nothing aborts: every failure is a returned status, and wlr_last_error gives a
 *     one-line message.  Device-side failures (a row system that is not positive
 *     definite, a rank-deficient X1) set an error word that the next synchronising
 *     call reports.
 */
#ifndef WLR_H
#define WLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WLR_OK = 0,
  WLR_ERR_INVALID_ARG = 1,        /* shape, k >= 1, k <= r <= min(m, n), null pointer  */
  WLR_ERR_NONPOSITIVE_WEIGHT = 2, /* some W1 entry <= 0 or not finite (Theorem 2)       */
  WLR_ERR_RANK_DEFICIENT = 3,     /* Cholesky of X1^T X1 broke down (Eq. 8 needs rank k)*/
  WLR_ERR_NOT_SPD = 4,            /* a row system diag(W1(i,:)^2) + C C^T broke down    */
  WLR_ERR_NO_CONVERGENCE = 5,     /* max_iter reached first: a warning, results valid   */
  WLR_ERR_DEVICE_TIMEOUT = 6,     /* a bounded device wait gave up                       */
  WLR_ERR_CUDA = 7,               /* a CUDA runtime call failed                          */
  WLR_ERR_OOM = 8,                /* device allocation failed                            */
  WLR_ERR_NOT_READY = 9,          /* call order: e.g. wlr_step before wlr_set_data       */
  WLR_ERR_UNSUPPORTED = 10        /* size outside what this build supports (k > 64 ...) */
} wlr_status;

typedef enum { WLR_F32 = 0, WLR_F64 = 1 } wlr_dtype;
typedef enum { WLR_MEM_DEVICE = 0, WLR_MEM_HOST = 1 } wlr_memory;

/* Arithmetic of the iteration.  FP64: every step in double.  FP32: float storage
 * and arithmetic, partial sums across thread blocks added in double. */
typedef enum { WLR_PREC_FP64 = 0, WLR_PREC_FP32 = 1 } wlr_precision;

/* Initial X1 (Algorithm 1, "Initialize (X1)_0"; Section 4.1 uses a random matrix). */
typedef enum {
  WLR_INIT_A1 = 0,      /* X1_0 = A1                                                    */
  WLR_INIT_RANDOM = 1,  /* X1_0 i.i.d. N(0,1): element (i,a), t = i + a*m, uses          */
                        /* SplitMix64(seed) outputs 2t, 2t+1 as u1, u2 = (x >> 11) 2^-53, */
                        /* z = sqrt(-2 ln(1 - u1)) cos(2 pi u2)  (Box-Muller)            */
  WLR_INIT_USER = 2     /* X1_0 given by the caller                                     */
} wlr_init;

/* Stopping rule of Section 4.1 with X_p = (X1_p, X1_p C_p + D_p) and
 * Error_p = ||X_{p+1} - X_p||_F. */
typedef enum {
  WLR_STOP_PAPER = 0,     /* Error_p < tol or Error_p / ||X_p||_F < tol              */
  WLR_STOP_RELATIVE = 1,  /* Error_p / ||X_p||_F < tol                               */
  WLR_STOP_NONE = 2,      /* run exactly max_iter iterations                          */
  WLR_STOP_OBJECTIVE = 3  /* |F_{p-1} - F_p| / F_p < tol (in-loop objective)          */
} wlr_stop;

typedef struct {
  int32_t precision;      /* wlr_precision (default FP32)                                */
  int32_t stop;           /* wlr_stop (default WLR_STOP_RELATIVE)                        */
  int32_t eig_block;      /* subspace block size b >= r-k for the rank-(r-k) SVD step;  */
                          /* 0 = min(n-k, 32, max(r-k+8, 2(r-k)))                      */
  int32_t eig_iters;      /* subspace iterations per sWLR iteration (warm start); 0 = 1 */
  int32_t eig_iters_cold; /* subspace iterations from a cold start; 0 = 40              */
  int32_t use_graph;      /* replay steady-state iterations as CUDA graphs (1): one     */
                          /* iteration per launch, three in wlr_solve with WLR_STOP_NONE */
  uint64_t seed;          /* seed of the random subspace start (and WLR_INIT_RANDOM)     */
  int32_t autotune;       /* 1: the row chunks of the per-iteration tensor-core Gram are  */
                          /* chosen by timing candidates at the first wlr_set_data of an  */
                          /* (m, n-k, k) shape in the process (cached; handles of one     */
                          /* shape share the choice, so they compute the same values);    */
                          /* 0 (default): a fixed rule (whole waves of CTAs on the SMs).  */
                          /* The paper has no counterpart.                                */
} wlr_options;

typedef struct wlr_handle_s* wlr_handle;

/* Fill *opt with the defaults listed above. */
void wlr_default_options(wlr_options* opt);

/* Create a solver for an m x n problem with k weighted columns and target rank r.
 * Requires 1 <= k <= 64, k <= r <= min(m, n), r - k <= 32.  opt may be NULL
 * (defaults).  cuda_stream is a cudaStream_t (NULL = the library creates its own).
 * Allocates all device workspace.  Returns WLR_ERR_INVALID_ARG / _UNSUPPORTED /
 * _OOM / _CUDA on failure, with *out set to NULL. */
wlr_status wlr_create(wlr_handle* out, int64_t m, int64_t n, int64_t k, int64_t r,
                      const wlr_options* opt, void* cuda_stream);

/* Attach the data of Eq. 5: A (m x n, leading dimension lda) and W1 (m x k,
 * leading dimension ldw), both of dtype dt in memory mem.  Runs the once-per-problem
 * setup: ||A2||_F^2 and K = A2^T A2 (the Gram of the unweighted frames, used to form
 * (P_perp A2)^T (P_perp A2) = K - B^T B each iteration).  Checks W1 > 0 and finite
 * (synchronises): WLR_ERR_NONPOSITIVE_WEIGHT otherwise. */
wlr_status wlr_set_data(wlr_handle h, const void* A, int64_t lda, const void* W1,
                        int64_t ldw, wlr_dtype dt, wlr_memory mem);

/* wlr_set_data with the weighted frames at arbitrary columns: cols (host, k distinct
 * indices in [0, n)) lists the columns of A that are weighted, in the order of W1's
 * columns.  Eq. 5 and Algorithm 1 take them as the first k columns; the library permutes A
 * to (A(:, cols), the other columns in increasing order) (a copy it owns for device data),
 * so X1 follows the order of cols and X2 that of the other columns; wlr_get_x returns
 * X = (X1, X2) in the caller's column order.  A later wlr_set_data resets the order to the
 * identity.  Errors as wlr_set_data, and WLR_ERR_INVALID_ARG for a bad index set. */
wlr_status wlr_set_data_cols(wlr_handle h, const void* A, int64_t lda, const void* W1,
                             int64_t ldw, wlr_dtype dt, wlr_memory mem, const int32_t* cols);

/* The whole approximation X (m x n, leading dimension ldx >= m, dtype dt, memory mem) in the
 * caller's column order: the weighted columns hold X1, the others X2 = X1 C + D with C, D
 * recomputed for the current X1 (Algorithm 1's output).  Synchronises. */
wlr_status wlr_get_x(wlr_handle h, void* X, int64_t ldx, wlr_dtype dt, wlr_memory mem);

/* Set X1_0 (Algorithm 1, initialisation).  X1_0 (m x k, leading dimension ldx, dtype
 * dt, memory mem) is read only for WLR_INIT_USER and may be NULL otherwise.  Resets
 * the iteration counter and the subspace warm start. */
wlr_status wlr_set_init(wlr_handle h, wlr_init kind, const void* X1_0, int64_t ldx,
                        wlr_dtype dt, wlr_memory mem, uint64_t seed);

/* One sWLR iteration (one pass of the loop body of Algorithm 1): from X1_p compute
 * C_p, D_p, the objective F_p = F(X1_p, C_p, D_p) (Eq. 8) and X1_{p+1}.  If
 * objective_out is non-NULL the call synchronises and stores F_p there (computed as
 * ||(A1-X1_p) o W1||^2 + ||A2||^2 - ||Q_p^T A2||^2 - sum of the r-k largest
 * sigma_j(P_perp A2)^2, i.e. the in-loop value). */
wlr_status wlr_step(wlr_handle h, double* objective_out);

/* Run Algorithm 1 from the current X1 until the stopping rule of the options holds
 * with threshold tol (Section 4.1 uses 1e-7) or max_iter iterations are done.
 * Synchronises.  *iters_out = iterations run, *objective_out = the last F_p (either
 * may be NULL).  Returns WLR_ERR_NO_CONVERGENCE (a warning; results valid) if
 * max_iter was reached with a rule other than WLR_STOP_NONE. */
wlr_status wlr_solve(wlr_handle h, double tol, int32_t max_iter, int32_t* iters_out,
                     double* objective_out);

/* F~(X1) = min_{C, rank-(r-k) D} F(X1, C, D) for the current X1, evaluated in FP64
 * with the residual ||A2 - X1 C - D||_F^2 summed entry by entry and the rank-(r-k)
 * SVD step iterated to convergence.  Synchronises.  For an FP32 handle this builds
 * (once) an FP64 copy of the problem. */
wlr_status wlr_objective(wlr_handle h, double* F_out);

/* Copy the current X1 (m x k) to X1 and, if X2 is non-NULL, X2 = X1 C + D
 * (m x (n-k)) with C, D recomputed for this X1 (the output of Algorithm 1).
 * dt/mem describe the destination buffers.  Synchronises when mem is host. */
wlr_status wlr_get_result(wlr_handle h, void* X1, int64_t ldx, void* X2, int64_t ldx2,
                          wlr_dtype dt, wlr_memory mem);

/* Factors of the last (C, D) step: C (k x (n-k)), V_s (the (n-k) x (r-k) right
 * singular vectors kept in D) and sigma2 (the r-k largest sigma_j(P_perp A2)^2).
 * Any pointer may be NULL.  Host memory, double precision, column-major.
 * Synchronises. */
wlr_status wlr_get_factors(wlr_handle h, double* C, double* Vs, double* sigma2);

/* Per-iteration history of the last wlr_solve / wlr_step calls since wlr_set_init:
 * F (in-loop objective F_p) and err (Error_p / ||X_p||_F, only with the paper or
 * relative stop rule; else NaN), up to cap entries each (host, may be NULL).
 * *count_out = entries available.  Synchronises. */
wlr_status wlr_get_history(wlr_handle h, double* F, double* rel_err, int32_t cap,
                           int32_t* count_out);

/* Iterations performed since wlr_set_init. */
wlr_status wlr_get_iteration(wlr_handle h, int32_t* p_out);

/* Checkpoint of the iteration, into host memory: the current X1_p, the factors of the
 * last (C, D) step that the next loop body of Algorithm 1 reads (C, Z2 = [C^T | V_s],
 * C C^T, C V_s, the Ritz values), the subspace basis and the R^{-1} that this build
 * carries from one iteration to the next, the iteration count and the history.  A handle
 * restored from it continues the same iteration bit for bit.  The paper has no
 * counterpart (its loop state is X1_p and p); the layout is private to this library and
 * versioned.  With buf == NULL only *size_out (bytes) is set; otherwise cap must be at
 * least that size (else WLR_ERR_INVALID_ARG).  WLR_ERR_NOT_READY before wlr_set_init.
 * Synchronises. */
wlr_status wlr_get_state(wlr_handle h, void* buf, int64_t cap, int64_t* size_out);

/* Restore a checkpoint made by wlr_get_state.  The handle must have the same m, n, k, r,
 * options and precision and must already hold the same data (wlr_set_data; the data is
 * not part of the state).  WLR_ERR_INVALID_ARG for a foreign, truncated or mismatched
 * buffer; WLR_ERR_NOT_READY before wlr_set_data.  Replaces any wlr_set_init.
 * Synchronises. */
wlr_status wlr_set_state(wlr_handle h, const void* buf, int64_t size);

/* FP64 refinement sweep: one loop body of Algorithm 1 (Section 3) from the handle's
 * current X1_p, computed in FP64 whatever the handle's precision (the data widened from
 * the handle's copy, thin QR by CholeskyQR2 in FP64, the rank-(r-k) truncation from an
 * eigensolve run until its values stop changing).  Writes X1_{p+1} to X1_out (m x k, FP64,
 * column-major, leading dimension ldx >= m, device or host memory per mem; NULL: not
 * written), F_p = F~(X1_p) to F_out and F~(X1_{p+1}) to F_next_out (each may be NULL).
 * The handle's own iterate, history and iteration count are not changed: the sweep ends
 * an FP32 solve with FP64 accuracy of the final step.  WLR_ERR_NOT_READY before
 * wlr_set_init; WLR_ERR_INVALID_ARG for ldx < m.  Synchronises. */
wlr_status wlr_refine(wlr_handle h, double* X1_out, int64_t ldx, wlr_memory mem, double* F_out,
                      double* F_next_out);

/* Batched solve: `iters` further iterations of Algorithm 1 (Section 3) on each of `count`
 * independent problems, which may differ in m, n, k, r and precision.  Each handle must
 * hold its data and an initial X1 (wlr_set_data, wlr_set_init).  The first iterations
 * after wlr_set_init run on each handle alone (the full-CholeskyQR warm-up and the cold
 * start of the subspace iteration); after that the iterations of all handles are joined
 * into one CUDA graph, with one child graph of three iterations per handle and no edges
 * between handles, and one graph launch advances every problem by three iterations.
 * Each handle computes exactly what wlr_solve(h, tol, iters, ...) computes with
 * WLR_STOP_NONE (no stopping test; the objective history is recorded).  Needs
 * use_graph = 1 on every handle for the joined launches; handles without it run alone.
 * handles: `count` distinct non-NULL handles (host array, borrowed); count == 0 is a
 * no-op.  failed_index (may be NULL): index of the handle whose error is returned, -1
 * if none or if the failure was not tied to one handle (its message is then on
 * handles[0]).  WLR_ERR_INVALID_ARG for a NULL or repeated handle, count < 0 or
 * iters < 0; WLR_ERR_NOT_READY when a handle lacks data or init; device errors of a
 * handle as wlr_step reports them.  Synchronises. */
wlr_status wlr_solve_batched(wlr_handle* handles, int32_t count, int32_t iters,
                             int32_t* failed_index);

/* Release the handle and all its device memory.  NULL is accepted. */
wlr_status wlr_destroy(wlr_handle h);

/* Static string for a status code. */
const char* wlr_status_string(wlr_status s);

/* Message of the last failing call on h (or of wlr_create when h is NULL). */
const char* wlr_last_error(wlr_handle h);

/* Measurement aid: run reps further sWLR iterations without CUDA graphs, each kernel
 * bracketed by CUDA events on the handle's stream, then (reps > 0, FP32) recompute the
 * setup Gram K = A2^T A2 once the same way (same values).  For up to max_kernels distinct
 * kernels: names ('\n'-separated, NUL-terminated, at most names_cap bytes), total
 * milliseconds and launch counts.  Advances the iterate like wlr_solve.  Synchronises. */
wlr_status wlr_profile(wlr_handle h, int32_t reps, char* names, int32_t names_cap,
                       double* ms_total, int32_t* launches, int32_t max_kernels,
                       int32_t* n_kernels);

/* Allocation-free X1 update.  The paper has no counterpart: this is a packaging of
 * the library's own row-update kernels for callers that cannot allocate device
 * memory -- code that must keep within memory it has already reserved (a framework
 * whose caching allocator owns the device), or latency-sensitive code for which a
 * cudaMalloc/cudaFree, which can synchronise the device, is not acceptable.
 *
 * Given X1_p (m x k, column-major, leading dimension m), the data A (m x n, lda) and
 * W1 (m x k, ldw), and the factors of the (C, D) step for X1_p -- C (k x (n-k),
 * leading dimension k) and V_s ((n-k) x (r-k), leading dimension n-k), as returned by
 * wlr_get_factors -- it writes X1_{p+1} (m x k, leading dimension m) with
 * X1_{p+1}(i,:) = E(i,:) (diag(W1(i,:)^2) + C C^T)^{-1},
 * E = A1 o W1 o W1 + (A2 - D) C^T, D = (P_perp A2) V_s V_s^T, i.e. the same values as
 * the X1 step of wlr_step.  All pointers are FP32 device pointers except wterm
 * (device double: ||(A1 - X1_p) o W1||_F^2, may be NULL) and status (device int, a
 * wlr_status code: WLR_OK, or WLR_ERR_NOT_SPD if a row system broke down, e.g. through a
 * non-finite weight, which this call does not check; may be NULL).  Work is queued on
 * cuda_stream (a cudaStream_t, NULL = the legacy default stream); the call does not
 * synchronise.
 *
 * Scratch: one fixed 1 MiB device array, held by every GPU that loads the library
 * until the process exits.  A problem fits when
 *   4 (n-k) ceil16(r) + 4 k^2 + 4 k (r-k) + 8 ceil(m / 64)  (each term rounded up to
 *   256 bytes, plus 256) <= 1 MiB,
 * e.g. m up to 5,000,000 with n - k <= 1000 and r <= 64; larger problems get
 * WLR_ERR_UNSUPPORTED.  No cudaMalloc, cudaFree or allocating routine is called.
 * The first call on a device (with that device current) looks up the array's device
 * address and sets kernel attributes; make that first call before any stream capture.
 * Every call on a device shares the one array and overwrites what the last call left
 * there, so calls whose GPU work overlaps (on different streams, or from different
 * threads) race: serialise them.
 * Returns WLR_ERR_INVALID_ARG (NULL pointer, shapes as in wlr_create, lda or ldw < m),
 * WLR_ERR_UNSUPPORTED (k > 64, r - k > 32, or the scratch rule above), WLR_ERR_CUDA; the
 * reason of a refusal is then in wlr_last_error(NULL).  With n = k (no unweighted frames)
 * C and Vs may be NULL. */
wlr_status wlr_x1_update_noalloc(const float* A, int64_t lda, const float* W1, int64_t ldw,
                                 const float* X1, int64_t m, int64_t n, int64_t k, int64_t r,
                                 const float* C, const float* Vs, float* X1_next,
                                 double* wterm, int* status, void* cuda_stream);

/* Self-test of the bounded device waits.  The paper has no counterpart: the tensor-core
 * kernels of this library wait on shared-memory barriers with a time limit (2 s), after
 * which they record an error bit and return, and the handle reports
 * WLR_ERR_DEVICE_TIMEOUT.  This call runs that same wait, limited to limit_ns (1 .. 2e9)
 * nanoseconds, on a barrier that nothing completes, on cuda_stream (NULL = the legacy
 * default stream), with no copy, MMA or tensor memory involved.  It returns
 * WLR_ERR_DEVICE_TIMEOUT when the wait gave up as designed (the expected result) and the
 * GPU context stays usable; WLR_OK would mean the limit did not work.  Synchronises. */
wlr_status wlr_selftest_bounded_wait(int64_t limit_ns, void* cuda_stream);

/* Number of kernels this handle has launched (graph replays count each node). */
int64_t wlr_kernel_launches(wlr_handle h);

/* ------------------------------------------------------------------------------------
 * Learned warm start.  Algorithm 1 starts from "Initialize (X1)_0" and Section 4.1 uses a
 * random matrix; the method itself never says where X1_0 comes from.  This build adds a
 * small network that predicts, from a downsampled clip and its weights, the span of the
 * solution X = (X1, X1 C + D), and starts from the weighted projection of A1 onto it:
 *
 *   input (per frame j, h x w):  channel 0 = block means of frame j / RMS of all of them,
 *                                channel 1 = block means of the per-pixel mean of W1's k
 *                                columns / their mean
 *   relu(conv 3x3 stride 2, 2 -> c1) -> relu(conv 3x3 stride 2, c1 -> c2) -> f_j (D values)
 *   z_j = [f_j | mean of f over the clip's frames] -> relu(fc1: 2D -> hidden) -> fc2 -> omega_j
 *   Omega (n x r_max) = the rows omega_j;  basis U = [A1 | 0] + A Omega(:, 1:r) / n
 *                                (m x r, full resolution: the weighted frames plus mixtures)
 *   X1_0(:, a) = U (U^T D_a U)^{-1} U^T D_a A1(:, a),  D_a = diag(W1(:, a)^2)
 *
 * The weighted projection minimises the first term of Eq. 5 over X1 with columns in
 * span(U).  That term keeps X1 close to A1, so the solution's span holds A1's columns up to
 * small corrections: the network predicts those corrections and the r - k other
 * directions.  Weights are kept in float (master copy, updated by Adam) and used in bfloat16
 * (round to nearest even) by every forward and backward kernel; all sums are float.
 * Training minimises ||P_Y - P_V||_F^2 / (2r), Y = U of the clip, against the column space
 * V of a converged solution (wlr_get_basis).  Network tensors are row-major:
 * X (frames, 2, h, w), Omega (frames, r_max).  Device pointers unless stated.
 * ------------------------------------------------------------------------------------ */
typedef struct wlr_ws_net_s* wlr_ws_net;

typedef struct {
  int32_t h, w;      /* network input frame size (downsampled), each >= 1               */
  int32_t c1, c2;    /* channels of the two convolutions                               */
  int32_t hidden;    /* width of the hidden fully-connected layer                      */
  int32_t r_max;     /* columns of Omega: ranks r <= r_max can be served                */
} wlr_ws_shape;

/* Network with weights N(0, 2/fan_in) from seed (SplitMix64 + Box-Muller as for
 * WLR_INIT_RANDOM, one stream per parameter index), biases 0, Adam moments 0.  max_frames
 * bounds the frames of one forward/backward call (activation buffers are allocated here).
 * stream: the cudaStream_t all of the network's work is queued on (NULL = the legacy
 * default stream); the calls that return host data or whose host arguments are copied
 * synchronise it.  WLR_ERR_INVALID_ARG for a bad shape. */
wlr_status wlr_ws_create(wlr_ws_net* out, const wlr_ws_shape* shape, int32_t max_frames,
                         uint64_t seed, void* stream);
wlr_status wlr_ws_destroy(wlr_ws_net net);
/* Number of parameters; the flat float layout is Wc1 (c1,2,3,3), b1, Wc2 (c2,c1,3,3), b2,
 * W3 (hidden, 2D), b3, W4 (r_max, hidden), b4, each row-major, D = c2 ceil(ceil(h/2)/2)
 * ceil(ceil(w/2)/2). */
int64_t wlr_ws_param_count(wlr_ws_net net);
/* Copy the float master weights (or the last gradients) out, or new master weights in (the
 * bfloat16 copy is refreshed), in the flat layout above; mem says host or device. */
wlr_status wlr_ws_get_params(wlr_ws_net net, float* out, wlr_memory mem);
wlr_status wlr_ws_get_grads(wlr_ws_net net, float* out, wlr_memory mem);
wlr_status wlr_ws_set_params(wlr_ws_net net, const float* in, wlr_memory mem);

/* Network input of one clip: A (m x n, column-major, lda >= m, float, device) with frames of
 * H x W pixels (m = H W, pixel index y W + x), W1 (m x k, ldw >= m); H = f h and W = f w for
 * an integer f.  Writes X (n, 2, h, w).  WLR_ERR_INVALID_ARG otherwise. */
wlr_status wlr_ws_prepare(wlr_ws_net net, const float* A, int64_t lda, const float* W1,
                          int64_t ldw, int32_t H, int32_t W, int32_t n, int32_t k, float* X);

/* Forward pass over `frames` frames of X that belong to consecutive clips: clip c holds
 * frames clip_start[c] .. clip_start[c+1]-1 (host array of nclips+1 entries, clip_start[0] =
 * 0, clip_start[nclips] = frames).  Writes Omega (frames x r_max) and keeps the activations
 * for wlr_ws_backward.  frames <= max_frames. */
wlr_status wlr_ws_forward(wlr_ws_net net, const float* X, int32_t frames,
                          const int32_t* clip_start, int32_t nclips, float* Omega);

/* Loss of one clip and its gradient: Y = [A1 | 0] + A Omega_c(:, 1:r) / n with A (m x n, lda),
 * A1 its first k columns, Omega_c (n x r_max, the clip's rows of Omega), V (m x r,
 * column-major, ldv >= m, orthonormal columns).  Adds ||P_Y - P_V||_F^2 / (2r) to *loss
 * (device double) and writes dOmega_c = d loss / d Omega_c (n x r_max; zero beyond column
 * r).  0 <= k <= r <= min(r_max, n). */
wlr_status wlr_ws_loss(wlr_ws_net net, const float* A, int64_t lda, int32_t m, int32_t n,
                       int32_t k, const float* Omega_c, int32_t r, const float* V, int64_t ldv,
                       double* loss, float* dOmega_c);

/* Backward pass of the last forward call: gradients of sum(dOmega o Omega) with respect to
 * every parameter, stored (not accumulated) as the net's gradients. */
wlr_status wlr_ws_backward(wlr_ws_net net, const float* dOmega);

/* One Adam step (Kingma & Ba 2015) on the stored gradients times grad_scale, step count
 * advanced by one; the bfloat16 copy is refreshed. */
wlr_status wlr_ws_adam(wlr_ws_net net, float lr, float beta1, float beta2, float eps,
                       float grad_scale);

/* Number of kernels the network object has launched. */
int64_t wlr_ws_launches(wlr_ws_net net);

/* Orthonormal basis (m x r, column-major, leading dimension ldv >= m, float, device) of the
 * column space of X = (X1, X1 C + D) at the handle's current iterate: the span of X1 and of
 * the r - k left singular vectors kept in D (Theorem 1), orthonormalised in double by
 * Cholesky QR twice.  WLR_ERR_NOT_READY before wlr_set_init.  Synchronises. */
wlr_status wlr_get_basis(wlr_handle h, float* V, int64_t ldv);

/* Initialise X1 from the network (replaces wlr_set_init): X = prepared input of the handle's
 * data (frames H x W, H W = m), Omega = forward pass, U = [A1 | 0] + A Omega(:, 1:r) / n,
 * then X1_0 the weighted projection above (Gram matrices and solves in double, with a ridge
 * of 1e-12 of the trace).  With fallback != 0 the objective F_0 = F(X1_0, C_0, D_0) of one
 * iteration from this start and from X1_0 = A1 (the value wlr_step returns) are compared and
 * the lower start is kept (A1 on a tie); *used_learned (may be NULL) says which.  Needs r <= r_max and n <= max_frames; resets the
 * iteration like wlr_set_init.  Float handles only.  Synchronises. */
wlr_status wlr_set_init_learned(wlr_handle h, wlr_ws_net net, int32_t H, int32_t W,
                                int32_t fallback, int32_t* used_learned);

#ifdef __cplusplus
}
#endif

#endif /* WLR_H */
