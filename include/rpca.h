/*
 * rpca.h -- C ABI of the GB300 robust-PCA solver (principal component pursuit
 * by the augmented-Lagrangian iteration) for ultrasound frame windows.
 *
 * Method (arXiv 2506.10257, Sec. II-A): a window of T frames of m pixels forms
 * the Casorati matrix X (m x T, Eq. 1 context).  PCP (Eq. 2) splits
 * X = L + S into a low-rank L (bound bubbles, tissue) and a sparse S (free
 * bubbles, noise).  Each iteration does
 *     Eq. 4  L = D_{1/mu}(X - S + Y/mu)        singular value thresholding
 *     Eq. 5  S = shrink_{lambda/mu}(X - L + Y/mu)
 *     Eq. 6  Y = Y + mu (X - L - S)
 * and stops when ||X - L - S||_F <= tol ||X||_F (Sec. II-A).
 *
 * Memory layout (all device buffers): frame-major, i.e. column-major X with
 * element (pixel p, frame t) at X[t*m + p]; frame t is a contiguous run of m
 * values.  Real data is float32; complex IQ data is interleaved complex64
 * (re, im) pairs with the same indexing.  Buffers must be 16-byte aligned.
 *
 * Ownership: the caller owns X, L, S and mask; X is only read.  A plan owns
 * its workspace (iterate state, Gram partials, eigenvectors) unless the
 * caller passes one.  Every entry point returns a status; nothing is thrown
 * across the ABI.  A plan is not thread-safe; a server is (submit/poll may be
 * called from several host threads).
 */
#ifndef RPCA_H_
#define RPCA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPCA_OK = 0,
  RPCA_NOT_CONVERGED = 1,   /* max_iter reached; outputs hold the last iterate */
  RPCA_PENDING = 2,         /* rpca_poll: request not finished yet */
  RPCA_ERR_ARG = -1,        /* invalid argument (shape, pointer, tolerance ...) */
  RPCA_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  RPCA_ERR_NOMEM = -3,      /* device allocation failed */
  RPCA_ERR_BUDGET = -4,     /* request exceeds the server's HBM budget */
  RPCA_ERR_TIMEOUT = -5,    /* a bounded device wait ran out */
  RPCA_ERR_NONFINITE = -6,  /* residual became NaN/Inf (input not finite) */
  RPCA_ERR_UNSUPPORTED = -7,/* shape/precision combination not built */
  RPCA_ERR_NOTFOUND = -8    /* unknown request id */
} rpca_status;

/* Element type of X, L, S.  R32: float32 envelope/RF data.  C64: complex64 IQ
 * data, (Re, Im) float pairs, frame-major; the SVT then acts on the Hermitian
 * Gram Z^H Z and the shrink of Eq. 5 on each entry's magnitude (phase kept).
 * C64 needs 2 T <= RPCA_MAX_T (the solver works on the interleaved real
 * embedding with 2 T columns), and 2 T <= 128 for the tensor-core precisions
 * (plans; batches of complex windows run FP32). */
typedef enum { RPCA_R32 = 0, RPCA_C64 = 1 } rpca_dtype;

/* Arithmetic of the two dense contractions per iteration (Z*Wbar and the
 * rotated Gram).  The eigensolve, the sigma-vs-tau decision, mu and the
 * convergence test are FP64 in every mode. */
typedef enum {
  RPCA_PREC_FP32 = 0,       /* FP32 CUDA-core FMA */
  RPCA_PREC_TF32X3 = 1,     /* tensor cores, TF32 hi/lo split, 3 products, FP32 accumulate */
  RPCA_PREC_BF16X3 = 2,     /* tensor cores, BF16 hi/lo split, 3 products, FP32 accumulate */
  RPCA_PREC_TF32 = 3        /* reserved: one plain TF32 product per contraction leaves L and S
                               about 7e-4 from the FP64 solution (262144 x 20 window), outside
                               the 1e-4 bound of the reduced precisions; plans reject it with
                               RPCA_ERR_UNSUPPORTED */
} rpca_precision;

/* Penalty schedule.  IALM: mu_1 = mu0_scale/||X||_2, mu_{k+1} = min(rho mu_k,
 * mu_max_factor mu_1).  FIXED_L1: mu = m T / (4 ||X||_1) for every iteration
 * (the choice of Sec. II-A / II-B). */
typedef enum { RPCA_MU_IALM = 0, RPCA_MU_FIXED_L1 = 1 } rpca_mu_schedule;

/* How the iterations are driven. */
typedef enum {
  RPCA_DRIVE_GRAPH = 0,     /* one CUDA graph per solve, device-side while loop, fused pass */
  RPCA_DRIVE_HOST = 1,      /* host loop, separate Gram / update passes, residual read back
                               every iteration (the plain form) */
  RPCA_DRIVE_STREAM = 2     /* the graph's kernels launched one by one on the stream, the host
                               reading the convergence flag every 8 iterations (for profilers
                               that cannot look inside a graph with a conditional node) */
} rpca_drive;

typedef struct {
  int64_t m;                /* pixels per frame (rows of X), >= 1 */
  int32_t T;                /* frames (columns of X), 1 <= T <= RPCA_MAX_T; precisions other
                               than FP32 need T <= 128 (real) or T <= 64 (complex) in plans,
                               T <= RPCA_MAX_T_NARROW (real) in batches */
  int32_t dtype;            /* rpca_dtype */
  int32_t precision;        /* rpca_precision */
  int32_t mu_schedule;      /* rpca_mu_schedule */
  int32_t drive;            /* rpca_drive */
  int32_t max_iter;         /* >= 1 (default 500) */
  double lambda;            /* <= 0 selects 1/sqrt(max(m, T)) */
  double mu0_scale;         /* IALM: mu_1 = mu0_scale / ||X||_2 (default 1.25) */
  double rho;               /* IALM growth factor (default 1.5), >= 1 */
  double mu_max_factor;     /* IALM cap mu_max = factor * mu0, mu0 the cold schedule's first
                               mu (default 1e7) */
  double tol;               /* relative Frobenius stopping tolerance (default 1e-7), > 0 */
  /* Warm start (the paper always starts from L = S = Y = 0; a sliding-window
   * stream can resume from the previous window's state instead).  With
   * warm_start = 1, on entry to rpca_solve the S buffer holds S0 and the L
   * buffer holds Y0 (m x T each); the first SVT then acts on
   * Z1 = X - S0 + Y0/mu1 (one extra Gram pass) and every later step is the
   * same iteration.  0 (default) ignores the buffers' contents. */
  int32_t warm_start;
  int32_t sharded;          /* 1: the window is split by pixel rows across processes and driven
                               step by step (rpca_step_*, below); default 0 */
  double mu_init;           /* > 0: first mu of the solve (default 0: the schedule's mu0) */
  double mu_prev_scale;     /* > 0 with warm_start and mu_init == 0: first mu = this times the
                               final mu of this plan's previous solve (default 0) */
} rpca_params;

/* Largest frame count.  Windows of T <= 32 frames run one pixel row per
 * thread; T in 33..224 run the shared-memory tiled path (FP32 only). */
#define RPCA_MAX_T 224
#define RPCA_MAX_T_NARROW 32

typedef struct {
  int32_t status;           /* rpca_status of this solve */
  int32_t iters;            /* completed iterations (Y updates) */
  int32_t rank;             /* singular values above 1/mu in the last iteration */
  int32_t sweeps;           /* Jacobi sweeps summed over the solve */
  double resid;             /* ||X - L - S||_F / ||X||_F of the last iteration */
  double mu;                /* penalty used by the last iteration */
  double normX;             /* ||X||_F */
  double lambda;            /* lambda used */
  double pass_us;           /* mean device time of the per-iteration passes after the
                               first (device global timer, first CTA start to last
                               CTA end), microseconds */
  double eig_us;            /* mean device time of the eigen-steps, microseconds */
  double init_us;           /* device time of the initial pass over X, microseconds */
  int32_t passes_timed;     /* passes in pass_us */
  int32_t eigs_timed;       /* eigen-steps in eig_us */
} rpca_result;

typedef struct rpca_plan_s* rpca_plan_t;

/* Fill *p with the defaults above for an m x T real window. */
rpca_status rpca_params_default(rpca_params* p, int64_t m, int32_t T);

/* Bytes of device workspace a plan with these parameters needs. */
rpca_status rpca_workspace_size(const rpca_params* p, size_t* bytes);

/* Create a plan.  `workspace` is a device buffer of at least
 * rpca_workspace_size() bytes owned by the caller (kept alive until
 * rpca_plan_destroy), or NULL to let the plan allocate its own.  Builds the
 * CUDA graph on first use.  Errors: RPCA_ERR_ARG, RPCA_ERR_UNSUPPORTED,
 * RPCA_ERR_NOMEM, RPCA_ERR_CUDA. */
rpca_status rpca_plan_create(const rpca_params* p, void* workspace, size_t workspace_bytes,
                             rpca_plan_t* out);

/* Solve PCP for one window on `stream` (a cudaStream_t, NULL = legacy default).
 *   X     device, m x T frame-major, read only.
 *   L, S  device outputs, m x T frame-major (may not alias X or each other).
 *   mask  optional device output of m bytes: 1 where the per-pixel temporal
 *         mean of |L| is >= theta (the binarised bound-bubble image of
 *         Sec. II-F), else 0.  NULL skips it.
 *   out   if non-NULL the call waits for the stream and fills *out; if NULL
 *         the call returns right after enqueueing and the result can be read
 *         with rpca_plan_result() after the stream has been synchronised.
 * Returns the solve status when out != NULL, else RPCA_OK once enqueued. */
rpca_status rpca_solve(rpca_plan_t plan, const void* X, void* L, void* S, uint8_t* mask,
                       float theta, void* stream, rpca_result* out);

/* Same as rpca_solve with HOST buffers: X_host (m*T values, frame-major) is
 * copied to device staging buffers owned by the plan (allocated on the first
 * call), the window is solved, and L, S (and the mask, if mask_host is not
 * NULL) are copied back into the host buffers; the call returns when they are
 * there.  Host buffers should be pinned (cudaHostAlloc) for full copy speed.
 * `out` may be NULL. */
rpca_status rpca_solve_host(rpca_plan_t plan, const void* X_host, void* L_host, void* S_host,
                            uint8_t* mask_host, float theta, void* stream, rpca_result* out);

/* Result of the last solve on this plan (call after synchronising its stream). */
rpca_status rpca_plan_result(rpca_plan_t plan, rpca_result* out);

/* Device-timer breakdown of the last solve (after synchronising its stream),
 * written to out[0..n): [0] mean eigen-step time in its control + load phase,
 * [1] in the Jacobi sweeps, [2] forming the rotation product, [3] basis update
 * and Wbar, all in microseconds; [4] Jacobi rounds executed per eigen-step;
 * [5] eigen-steps timed; [6] mean per-iteration pass time until the last CTA
 * has written its partial sums, [7] in the first-level cross-CTA reduction,
 * [8] in the final reduction (microseconds).  Entries past 9 are left
 * untouched.  Implementation instrumentation: the paper has no counterpart. */
rpca_status rpca_plan_timings(rpca_plan_t plan, double* out, int32_t n);

void rpca_plan_destroy(rpca_plan_t plan);

const char* rpca_status_str(int32_t status);

/* ---- batched persistent form --------------------------------------------- */

/* Many independent windows (each its own Casorati matrix, Sec. II-A, with its
 * own m, T and parameters) solved by one persistent cooperative launch,
 * captured in a CUDA graph: every window runs the same iteration as
 * rpca_solve (Eq. 4-6, stopping test of Sec. II-A), so each result equals the
 * window's single solve within the precision's tolerance.  The paper solves
 * one window at a time; batching is this library's throughput form. */
typedef struct rpca_batch_s* rpca_batch_t;

/* Device buffers of one window of a batch, laid out as in rpca_solve. */
typedef struct {
  const void* X;    /* m x T frame-major, read only, 16-byte aligned */
  void* L;          /* m x T, written (also the first dual buffer during the solve) */
  void* S;          /* m x T, written */
  uint8_t* mask;    /* m bytes or NULL: temporal mean |L| >= theta */
  float theta;
  int32_t pad_;
} rpca_window;

/* Creates a batch of n windows with parameters params[0..n) (copied).  The
 * batch owns one workspace per window (rpca_workspace_size bytes each) and the
 * launch descriptor.  Every window has the same precision: RPCA_PREC_FP32, or
 * RPCA_PREC_TF32X3 / RPCA_PREC_BF16X3 for real windows of <= 32 frames (the
 * two contractions of each iteration's pass on the tensor cores, as in
 * rpca_solve); other combinations return RPCA_ERR_UNSUPPORTED.  drive is
 * ignored.  The CTA schedule is the one tuned
 * before for the same window shapes in this process (rpca_batch_tune), else a
 * default (paired lanes of two windows each, CTAs proportional to m*T). */
rpca_status rpca_batch_create(const rpca_params* params, int32_t n, rpca_batch_t* out);

/* Solves windows win[0..n) in one launch on `stream`.  With out != NULL
 * (n entries) the call waits and fills each window's rpca_result, returning the
 * worst status (negative first); with out == NULL it returns at once.  The
 * window buffers must stay alive until the stream reaches the launch's end. */
rpca_status rpca_batch_solve(rpca_batch_t batch, const rpca_window* win, void* stream, rpca_result* out);

/* Autotuner: times every candidate schedule (lanes, CTA share exponent, CTAs
 * per SM, paired or not) on these windows, `reps` timed solves each (median), keeps the
 * fastest for this batch and for later batches of the same shapes in this
 * process.  *best_ms (nullable) gets its median time per solve.  Synchronous. */
rpca_status rpca_batch_tune(rpca_batch_t batch, const rpca_window* win, void* stream, int32_t reps,
                            double* best_ms);

/* Sets the schedule by hand (as rpca_batch_tune would pick one): `lanes`
 * lanes (capped at the resident CTAs), lane CTAs ~ load^alpha, ctas_per_sm
 * resident CTAs per SM (1 .. the kernel's maximum, info[4]), paired 0/1.
 * Waits for the batch's launch in flight.  Errors: RPCA_ERR_ARG. */
rpca_status rpca_batch_set_schedule(rpca_batch_t batch, int32_t lanes, double alpha, int32_t ctas_per_sm,
                                    int32_t paired);

/* Schedule in use: info[0..n) = {grid CTAs, lanes, CTAs per SM,
 * 1000 * share exponent, max resident CTAs per SM, graph captured (0/1),
 * paired lanes (0/1)}.  Paired lanes (the default for two or more windows):
 * a lane of two or more windows runs them two at a time, its last CTA running
 * every eigen-step (one window's) while its other CTAs run the other window's
 * pass, so the one-CTA eigen-steps overlap the passes. */
rpca_status rpca_batch_info(rpca_batch_t batch, int32_t* info, int32_t n);

/* CTAs each window uses (n >= number of windows). */
rpca_status rpca_batch_window_ctas(rpca_batch_t batch, int32_t* ctas, int32_t n);

/* The batch form's CTA schedule as a pure host computation (no device call),
 * for inspecting a schedule before creating a batch.  Windows go to lanes
 * (contiguous CTA ranges that run their windows one after another) by
 * longest-processing-time first on m[w] * T[w], equal loads in index order;
 * L = min(lanes, n, ctas) lanes; lane l gets CTAs proportional to (its load)^alpha,
 * at least one and at most the largest max_ctas[w] of its windows (NULL: no
 * limit), summing to at most `ctas`, fractional shares settled by largest
 * remainders.  rpca_batch_create and rpca_batch_tune build their schedules
 * with this computation (ctas = SMs x CTAs per SM, max_ctas the windows' useful
 * CTA counts).  Outputs: *n_lanes = L; lane_ctas[0..L) the lanes' CTAs;
 * order[0..n) the windows in lane order, lane l running order[lane_end[l-1] ..
 * lane_end[l]) (lane_end[-1] = 0) in descending load; lane_ctas and lane_end
 * need n entries.  Errors: RPCA_ERR_ARG (n < 1, a null pointer other than
 * max_ctas, ctas < 1, lanes < 1, alpha negative or not finite, an m, T or
 * max_ctas entry < 1). */
rpca_status rpca_batch_schedule(int32_t n, const int64_t* m, const int32_t* T, const int32_t* max_ctas,
                                int32_t ctas, int32_t lanes, double alpha, int32_t* n_lanes, int32_t* lane_ctas,
                                int32_t* order, int32_t* lane_end);

/* rpca_batch_solve with HOST buffers: win[i].X, L, S and mask are host
 * pointers (pinned host memory, cudaHostAlloc, for full copy speed; mask may
 * be NULL), laid out as the device buffers of rpca_solve.  The batch owns two
 * device staging sets (one per call parity, allocated on the first call) and
 * two copy streams: a call uploads every X into its set (after the downloads
 * of the call two before it have landed), solves the set on `stream` in one
 * persistent launch, and downloads L, S and the masks.  Consecutive calls
 * therefore overlap one call's uploads and the previous call's downloads with
 * the solves.  With out != NULL the call waits until its own downloads (and
 * those of every earlier call) have landed and fills out[0..n) as
 * rpca_batch_solve does, returning the worst status; with out == NULL it
 * returns once enqueued, and the host buffers of every call made so far must
 * stay untouched until a later call with out != NULL returns.  Errors:
 * RPCA_ERR_ARG (null pointers), RPCA_ERR_NOMEM (staging allocation),
 * RPCA_ERR_CUDA. */
rpca_status rpca_batch_solve_host(rpca_batch_t batch, const rpca_window* win, void* stream, rpca_result* out);

void rpca_batch_destroy(rpca_batch_t batch);

/* ---- served form ----------------------------------------------------------- */

/* A request loop over sliding frame windows from several probes (the paper's
 * real-time goal, Sec. I and IV; the serving machinery itself has no
 * counterpart in the paper).  Each request is one window solved exactly as by
 * rpca_solve on a plan of its parameters, except that a probe's windows after
 * its first may warm-start (see rpca_server_set_warm).
 *
 * Continuous batching: requests queue in arrival order and start as soon as a
 * slot (one of max_slots CUDA streams) is free and their probe's device state
 * fits the budget, while earlier solves are still running; solves of
 * different probes overlap on the device.  A probe's windows run in arrival
 * order.  Progress happens inside rpca_submit, rpca_poll, rpca_server_wait and
 * rpca_server_stats (no background thread).
 *
 * Memory: per probe the server holds a plan workspace (rpca_workspace_size)
 * and the probe's S and Y state (2 m T floats); that total is charged against
 * hbm_budget_bytes.  Idle probes (nothing queued or running) are evicted,
 * least recently used first, when a new probe needs room; their next window
 * starts cold.  The caller's X, L, S buffers are not charged. */
typedef struct rpca_server_s* rpca_server_t;

/* max_slots in [1, 256].  Defaults: warm start off (every window a cold
 * solve), warm_mu_scale 0.1, cold_every 0. */
rpca_status rpca_server_create(size_t hbm_budget_bytes, int32_t max_slots, rpca_server_t* out);

/* Warm-start policy.  warm = 1: a probe's window k+1 (assumed to be window k
 * shifted by one frame) starts from S0, Y0 = window k's final S, Y with the
 * oldest frame dropped and a zero frame appended, and first mu =
 * warm_mu_scale * window k's final mu (warm_mu_scale = 0: the schedule's mu0).
 * cold_every = n > 0 makes every n-th window of a probe start cold (bounds the
 * drift of a long warm chain); 0 never.  warm = 0 (the default): every window
 * starts cold.  A warm start saves iterations (about 34 -> 7 at
 * warm_mu_scale 0.1 on 20-frame windows) but the stopping test of Sec. II-A
 * bounds the primal residual only, so the solve ends at a point that depends
 * on its start: measured on a 40-window chain of 96 x 96 x 20 windows with
 * the oracle, bound-bubble mask Dice against each window's cold solve falls
 * to 0.91 (warm_mu_scale 0.1), 0.94 (1e-3), 0.99 (0 = cold mu schedule). */
rpca_status rpca_server_set_warm(rpca_server_t server, int32_t warm, double warm_mu_scale, int32_t cold_every);

/* Queue one window (device buffers as in rpca_solve; they must stay alive and
 * untouched until the request is reported done) for probe `stream_key`.
 * *req_id identifies it.  RPCA_ERR_BUDGET when the probe's state alone
 * exceeds the budget; parameter errors as rpca_plan_create.  warm_start,
 * mu_init and mu_prev_scale of *p are ignored (the server's policy rules). */
rpca_status rpca_submit(rpca_server_t server, const rpca_params* p, const void* X, void* L, void* S,
                        uint8_t* mask, float theta, int32_t stream_key, uint64_t* req_id);

/* RPCA_PENDING while the request is queued or running; once done, fills *out
 * (nullable), forgets the request and returns its status.  RPCA_ERR_NOTFOUND
 * for an unknown (or already reported) id. */
rpca_status rpca_poll(rpca_server_t server, uint64_t req_id, rpca_result* out);

/* Blocks until the request is done, then as rpca_poll.  RPCA_ERR_BUDGET if it
 * is queued with nothing running that could free memory for it. */
rpca_status rpca_server_wait(rpca_server_t server, uint64_t req_id, rpca_result* out);

/* stats[0..n) = {bytes held, peak bytes held, budget, queued, running, peak
 * running, started, finished, probes evicted, requests refused}. */
rpca_status rpca_server_stats(rpca_server_t server, int64_t* stats, int32_t n);

/* Waits for running solves, frees every probe's state. */
void rpca_server_destroy(rpca_server_t server);

/* ---- kernel-level entry points (each one step of the iteration) ---------- */

/* Rotated Gram of a window: G = (Z V)^T (Z V) with Z = X (frame-major m x T,
 * real float32) and V a T x T row-major float32 matrix (NULL = identity).
 * G is written as T x T row-major float64 on the device.  This is the
 * contraction that feeds the SVT step of Eq. 4 (SVD of Z through the
 * eigen-decomposition of its Gram).  T <= RPCA_MAX_T_NARROW.  Synchronous on
 * `stream`. */
rpca_status rpca_gram(const float* X, int64_t m, int32_t T, const float* V, double* G,
                      int32_t precision, void* stream);

/* Symmetric eigen-decomposition of a T x T float64 matrix G (row-major,
 * device) by cyclic Jacobi in FP64 on one CTA: on return evals[i] and the
 * columns of evecs (T x T row-major, device) satisfy G evecs = evecs diag(evals),
 * evals in descending order.  T <= RPCA_MAX_T_NARROW.  Synchronous on `stream`. */
rpca_status rpca_eig(const double* G, int32_t T, double* evals, double* evecs, void* stream);

/* ---- entry point that allocates no device memory ------------------------ */

/* The paper has no counterpart to this entry point; it serves callers that may
 * not allocate device memory once they are running: a real-time scanner
 * pipeline that reserves all device memory at start-up and must not block on
 * cudaMalloc (which can synchronise the whole device) while frames stream in,
 * or a process whose device memory belongs to another framework's pool.
 *
 * Computes the same G = (Z V)^T (Z V) as rpca_gram (Z = X, frame-major m x T
 * real float32 on the device; V row-major T x T float32 on the device or NULL
 * for the identity; G row-major T x T float64 on the device, written by the
 * call), but asynchronously on `stream` and with no cudaMalloc, cudaFree or
 * other allocating call: its scratch (about 2.4 MB: partial Grams of at most
 * 512 CTAs, reduction counters, control block) is a fixed array compiled into
 * the library, one copy on every GPU that loads it, held until the process
 * exits.  The caller still provides X, V and G.
 *   - T must be <= RPCA_MAX_T_NARROW (else RPCA_ERR_UNSUPPORTED); m is not limited
 *     (the CTAs stride over the pixels).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is looked up again when the
 *     device's current context has changed since (for instance after
 *     cudaDeviceReset), so make the first call after such a change outside
 *     stream capture too.
 *   - Every call shares the one array and clears its counters first; calls
 *     whose work overlaps on the GPU (other streams, other host threads) race
 *     on it and must be serialised by the caller.
 *   - G is valid once `stream` has been synchronised. */
rpca_status rpca_gram_noalloc(const float* X, int64_t m, int32_t T, const float* V, double* G, void* stream);

/* ---- one window split by pixel rows across processes ----------------------- */

/* The method's only exchange is through the T x T Gram (Eq. 4 through the
 * eigen-decomposition of Z^T Z): with the pixel rows of one window spread over
 * several processes (one GPU each), every process runs the pass over its own
 * rows, the processes sum the Gram and the residual sums (an all-reduce of
 * T*32 + 2 doubles per iteration), and every process then runs the
 * same eigen-step on the same sums, so the iteration is the one of the whole
 * window.  A plan created with params.sharded = 1 (real FP32, T <=
 * RPCA_MAX_T_NARROW, IALM schedule, no warm start; params.lambda set from the
 * whole window: 1/sqrt(max(m_total, T)); params.m = this process's rows)
 * exposes the steps:
 *   rpca_step_begin  binds this call's X, L, S (this process's rows, frame-major
 *                    m x T, 16-byte aligned) and mask/theta as rpca_solve does;
 *   rpca_step_run    launches one step: RPCA_STEP_INIT (the norms and Gram of X),
 *                    RPCA_STEP_EIG_INIT (mu0 and the first eigen-step),
 *                    RPCA_STEP_PASS (the fused pass of an iteration),
 *                    RPCA_STEP_EIG (residual test, mu update, eigen-step),
 *                    RPCA_STEP_FINAL (L and the mask);
 *   rpca_step_sums   device pointers of the sums to reduce after RPCA_STEP_INIT and
 *                    RPCA_STEP_PASS: the Gram (T rows of 32 doubles, row stride 32,
 *                    columns >= T zero; FP64 sums of the CTAs' FP32 partials) and
 *                    {e2, l1} (2 doubles);
 *   rpca_step_done   synchronises `stream` and reports whether the solve has
 *                    ended (and its result, when `out` is not NULL).
 * Order: begin, INIT, reduce, EIG_INIT, then while not done: PASS, reduce, EIG;
 * then FINAL.  A plan with sharded = 1 also solves a whole window with
 * rpca_solve.  Errors: RPCA_ERR_ARG (NULL plan or pointers, a plan without
 * sharded = 1, an unknown step), RPCA_ERR_CUDA (a launch failed). */
typedef enum {
  RPCA_STEP_INIT = 0,
  RPCA_STEP_EIG_INIT = 1,
  RPCA_STEP_PASS = 2,
  RPCA_STEP_EIG = 3,
  RPCA_STEP_FINAL = 4
} rpca_step;
rpca_status rpca_step_begin(rpca_plan_t plan, const float* X, float* L, float* S, uint8_t* mask, float theta,
                            void* stream);
rpca_status rpca_step_run(rpca_plan_t plan, int32_t step, void* stream);
rpca_status rpca_step_sums(rpca_plan_t plan, double** gram, double** sums);
rpca_status rpca_step_done(rpca_plan_t plan, int32_t* done, rpca_result* out, void* stream);

/* ---- frame pre-filter of the in vivo reference ---------------------------- */

/* Before its 132-frame reference solve (Sec. III, "Applying the RPCA method")
 * the paper excludes the frames whose correlation with their neighbouring
 * frames is below 0.8 and applies a temporal moving average over 20 frames.
 * rpca_prefilter does both on the device, stream-ordered, with no host round
 * trip, so its output can feed rpca_solve on the same stream.  Readings (the
 * paper gives no formula): the correlation of frames t and t+1 is Pearson's
 * coefficient over all m pixels (a frame without variance correlates 0);
 * frame t is kept when it correlates at or above corr_min with at least one
 * neighbour (frames t-1, t+1; a window of one frame keeps it); the moving
 * average covers whole windows of kept frames only: output frame j is the
 * mean of kept frames j .. j+window-1, j = 0 .. K-window (K kept frames).
 *   X       frame-major T x m float32 on the device (frame t at X + t*m), read only.
 *   Y       device, room for max(T - window + 1, 0) frames of m floats (frame-major);
 *           the first count[1] frames are written.
 *   kept    device int32[T]: the kept frame indices, increasing (first count[0]).
 *   count   device int32[2]: {K, max(K - window + 1, 0)}.
 *   corr    device float64[T - 1] (nullable): the neighbour correlations,
 *           corr[t] between frames t and t+1.
 *   scratch device memory of rpca_prefilter_scratch_bytes(m, T) bytes, owned by
 *           the caller, not shared with a call in flight.
 * Correlations are accumulated in FP64 (FP32 inputs make every product exact);
 * the window sums slide in FP64.  Errors: RPCA_ERR_ARG (a null pointer, m < 1,
 * T < 1, window < 1, corr_min NaN, X or Y not 4-byte aligned),
 * RPCA_ERR_UNSUPPORTED (T > 65535), RPCA_ERR_CUDA (a launch failed).  The
 * outputs are valid once `stream` has reached the call. */
size_t rpca_prefilter_scratch_bytes(int64_t m, int32_t T);
rpca_status rpca_prefilter(const float* X, int64_t m, int32_t T, double corr_min, int32_t window, float* Y,
                           int32_t* kept, int32_t* count, double* corr, void* scratch, void* stream);

/* Temporal high-pass variant of rpca_prefilter.  Sec. IV suggests a
 * high-pass temporal filter before RPCA to take out slowly varying background
 * motion, without defining one; it is read here as the complement of the
 * moving average above: output frame j is kept frame j + h minus the mean of
 * kept frames j .. j+window-1, h = (window - 1) / 2 rounded down (the window's
 * centre for odd window), so what is constant or linear in time over a window
 * (odd window) is removed.  Same arguments, outputs, frame exclusion, scratch
 * and errors as rpca_prefilter; Y receives the high-passed frames (the
 * difference formed in FP64, rounded once to FP32). */
rpca_status rpca_prefilter_highpass(const float* X, int64_t m, int32_t T, double corr_min, int32_t window,
                                    float* Y, int32_t* kept, int32_t* count, double* corr, void* scratch,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RPCA_H_ */
