/*
 * tikh.h -- C-ABI of the GB300 superfast Tikhonov solver.
 *
 * Solves the l2-penalised Tikhonov problem of Turnes, Balcan & Romberg, "Superfast Tikhonov
 * Regularization of Toeplitz Systems" (arXiv 1302.6945):
 *
 *     x = argmin_x ||T x - b||^2 + lambda ||x||^2 = (T^H T + lambda I)^{-1} T^H b      (Eq. (tik), (tiksol))
 *
 * for an m x n Toeplitz T = [a_{i-j}] (Sec. 2, l2-norm penalisation with L = beta I, lambda = |beta|^2),
 * by the extension-and-transformation of Sec. 3-4.1 and the divide-and-conquer tangential
 * interpolation of Sec. 4.3-6 (Algorithm 1 with paired interleaving, Algorithm 2 sizing).
 * Every arithmetic step runs in CUDA kernels on the plan's stream.
 *
 * Conventions
 *  - col[d] = a_d (d = 0..m-1, first column of T); row[d] = a_{-d} (d = 1..n-1, first row of T;
 *    row[0] is ignored).
 *  - TIKH_R64: col, row, b, x are real float64 arrays; TIKH_C128: interleaved complex128 (re, im).
 *  - Pointers passed to tikh_solve / tikh_solve_normal are DEVICE pointers, caller-owned, contiguous,
 *    16-byte aligned, valid until the stream reaches the end of the call's work.  tikh_solve_host
 *    takes HOST pointers and copies through the plan's staging buffers.
 *  - The plan owns all device workspace; nothing else is allocated per call.
 *  - lambda must be finite and > 0.  m, n >= 1; m < n is solved through the identity
 *    (T^H T + lambda I)^{-1} T^H b = T^H (T T^H + lambda I)^{-1} b on the tall matrix T^H.
 *
 * Errors: every int-returning call returns TIKH_OK (0) or a negative TIKH_E* code; nothing aborts,
 * traps or exits.  Device-side failures are recorded in the plan's status word and returned by the
 * next synchronising call (tikh_solve, tikh_solve_host, tikh_sync).
 */
#ifndef TIKH_H
#define TIKH_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define TIKH_OK 0
#define TIKH_EINVAL (-1)        /* bad argument (sizes, lambda, dtype, null pointer) */
#define TIKH_ENOMEM (-2)        /* device or host allocation failed */
#define TIKH_ECUDA (-3)         /* a CUDA runtime call failed */
#define TIKH_ENUMERIC (-4)      /* final tau-degree pattern is not one 0 and four 1s, or a non-finite value */
#define TIKH_EDIFFICULT (-5)    /* more deferred (difficult) conditions than the plan can hold */
#define TIKH_ENOTCONVERGED (-6) /* iterative refinement did not reach its tolerance */
#define TIKH_ETIMEOUT (-7)      /* a bounded device wait gave up */
#define TIKH_EDEGREE (-8)       /* a basis degree exceeded its planned transform length (retried internally) */

typedef enum { TIKH_R64 = 0, TIKH_C128 = 1 } tikh_dtype;
/* Precision of the solve (the pattern of Sec. 7.2's refinement remark, made concrete):
 *  TIKH_PREC_FP64         every step in FP64 (the plain method).
 *  TIKH_PREC_FP32         the O(N log^2 N) part of the recursion -- the FFT-form evaluations of B_L at the
 *                         right child's nodes with their residual updates, and the FFT-form basis products
 *                         (Alg. 1 steps 2 and 4) -- runs in FP32 (complex64 transforms, FP32 pointwise
 *                         products and accumulation).  FP64 stays for the leaves (the serial single-point
 *                         construction, its pivot and deferral decisions), the tau-degree bookkeeping, the
 *                         small-node direct forms, the stored basis and residual rows, the length-N transforms
 *                         of the extension and the refinement residual.  Less accurate (the error of one
 *                         solve is far above the FP64 method's); opts.refine_steps corrections as in FP64.
 *  TIKH_PREC_FP32_REFINE  TIKH_PREC_FP32 solves plus iterative refinement with the FP64 residual
 *                         r = y - (T^H T + lambda I) x computed by FP64 FFT matrix-vector products (Sec. 7.3);
 *                         opts.refine_steps corrections (0 -> 2), each an FP32-stage solve. */
typedef enum { TIKH_PREC_FP64 = 0, TIKH_PREC_FP32_REFINE = 1, TIKH_PREC_FP32 = 2 } tikh_prec;

typedef struct tikh_plan_s* tikh_plan;
typedef struct tikh_batch_plan_s* tikh_batch_plan;

/* Planner options (NULL -> defaults).
 *  n_lim     leaf cutoff N_lim (Sec. 6.2): leaves hold at most 2M <= n_lim (+ rounding) conditions.
 *            Default 32; valid 4..64.  Large serial leaves lose accuracy.
 *  m_min     lower bound on M in Algorithm 2 (forces a larger extension k); 0 = none.
 *  fill      extension entries "similar in value" (Sec. 6.2): 0 = seeded pseudo-random of the
 *            coefficients' size (default), 1 = linear ramp between a_{m-1} and a_{-(n-1)}.
 *  eps_diff  difficult-point threshold (Sec. 5): a leaf defers its remaining conditions when the
 *            best one has |r_pivot| < eps_diff ||r||_2.  Default 1e-8.
 *  max_difficult  capacity of the deferred-condition list (default 4096).
 *  refine_steps   iterative-refinement corrections after the direct solve (default 0 = the plain
 *            method; 0..8).  Each correction recomputes r = y - (T^H T + lambda I) x by FFT matrix-
 *            vector products (Sec. 7.3) and solves for the correction with the same algorithm
 *            (Sec. 7.2: the result "can be further improved with iterative refinement").
 *  batch     largest number of same-shape problems per tikh_solve_strided call (default 1); the
 *            plan's workspace scales with it.
 *  graph     1: tikh_solve / tikh_solve_async / tikh_solve_strided capture the whole solve (every
 *            kernel of every recursion node) into one CUDA graph on the first call with a given number of
 *            problems and replay it for every later such call (the kernels read each call's pointers,
 *            sizes and lambdas from device tables written before the replay); 0 (default): stream
 *            launches.  Not used with profiling on.
 *  prod_direct_max  step-4 products (Alg. 1) of planned length P <= this are computed directly
 *            (schoolbook, one warp per output coefficient), longer ones by FFT; 0 (default): automatic
 *            (360 for batch = 1, where a small node is latency-bound; smaller for batches, where the
 *            O(P^2) direct product is FP64-throughput-bound).  0..4096.
 *  eval_direct_max  step-2 evaluations of B_L at <= this many nodes per coset are computed directly
 *            (chunked Horner), larger ones by FFT; 0 (default): automatic (80 for batch = 1).  0..4096.
 *  refine_tol  with refine_steps > 0: after the last correction, a relative residual
 *            ||y - (T^H T + lambda I) x|| / ||y|| above refine_tol makes the call return TIKH_ENOTCONVERGED
 *            (x is still written).  0 (default): no check.
 *  fft_radix  largest power-of-two radix of the FFT stages: 8 (default, 0) or 4 (more, lighter stages).
 *  fft_tile   elements per CTA for transforms shorter than it (several transforms share a CTA): a power
 *            of two up to 4096; 0 = 256.  Both are tuning knobs (tikh.autotune); the results agree to rounding.
 *  wait_polls  bound on the one in-kernel wait (the leaf's basis-rebuild warps polling for the next
 *            pivot step): after this many polls the wait gives up and the call returns TIKH_ETIMEOUT.
 *            0 (default): 2^24 polls.  0..2^30.  A small value exists to exercise the failure path.
 */
typedef struct {
  int n_lim;
  int m_min;
  int fill;
  double eps_diff;
  int max_difficult;
  int refine_steps;
  int batch;
  int graph;
  int prod_direct_max;
  int eval_direct_max;
  int wait_polls;
  double refine_tol;
  int fft_radix;
  int fft_tile;
} tikh_opts;

typedef struct {
  int64_t N, M, k; /* nodes N = 2^p M, extension k = N - (m+n-1) of the core (tall) problem */
  int p;           /* paired-interleaving splits; 2^p leaves */
  int dual;        /* 1: m < n solved through T^H */
  int64_t n_difficult; /* conditions deferred to the end in the last solve */
  int delta[7];        /* final tau-degrees of the basis columns in the last solve (5 used; 7 for the general
                        * problem) */
  int jstar;           /* column holding the solution */
  int retries;         /* internal re-runs after TIKH_EDEGREE */
  int64_t kernel_launches; /* kernels enqueued by the last solve */
  int64_t workspace_bytes; /* device bytes owned by the plan */
  int refine_steps;        /* corrections applied in the last solve */
  double rel_residual;     /* largest ||y - (T^H T + lambda I) x|| / ||y|| after refinement (-1 if none) */
  int batch;               /* problems in the last call */
  double prof_leaf_ms;     /* with profiling on: summed duration of the leaf launches since it was switched on */
  int64_t prof_leaf_launches; /* with profiling on: leaf launches timed since it was switched on */
  int graph;                  /* 1 if the last solve ran as a (captured or replayed) CUDA graph */
  /* with profiling flag 2: summed event-timed duration and count of the schedule's launch groups since
   * profiling was switched on, by kind: [0] leaves, [1] evaluations (Sec. 6.1 updates of a right
   * child's conditions), [2] basis products, [3] the rest (transform, conditions, difficult points,
   * extraction, refinement, output) */
  double prof_kind_ms[4];
  int64_t prof_kind_count[4];
  /* algorithmic FLOPs of one problem's core solve by the same kinds (a model of the arithmetic the
   * method needs: 5 L log2 L per complex FFT of length L, 8 per complex multiply-add; see the plan's
   * documentation), and the part of them the FFT stages run in FP32 (0 for TIKH_PREC_FP64).  A refined
   * solve runs the core solve 1 + refine_steps times. */
  double model_flops[4];
  double model_flops_fp32[4];
  double last_correction;  /* largest ||dx|| / ||x|| of the last refinement correction over the call (-1 if none):
                            * an estimate of the error of the solution before that correction */
} tikh_stats;

typedef struct {
  int ngroups;             /* groups of problems sharing N (and the m < n form): one schedule each */
  int max_waves;           /* most sequential waves of any group (items beyond the workspace budget) */
  int64_t items;           /* (problem, lambda) pairs per call = nprob * nlambda */
  int64_t kernel_launches; /* kernels enqueued per call (all groups) */
  int64_t workspace_bytes; /* device bytes owned by the batch plan */
  int graph;               /* 1 if the last call ran as one captured CUDA graph */
  int retries;             /* re-runs after TIKH_EDEGREE in the last call */
  int64_t n_difficult;     /* deferred conditions in the last wave of every group, summed */
  double rel_residual;     /* largest refinement residual over the last wave of every group (-1: none) */
  double last_correction;  /* largest ||dx|| / ||x|| of the last correction, same items (-1: none) */
  /* algorithmic FLOPs of one core solve of every item of a call, by kind (leaf, evaluation, product,
   * other) as in tikh_stats, and their FP32-stage part */
  double model_flops[4];
  double model_flops_fp32[4];
  /* with profiling on (tikh_batch_set_profiling): event-timed durations and counts of the launch groups
   * by kind, summed over the groups of every call since profiling was switched on */
  double prof_kind_ms[4];
  int64_t prof_kind_count[4];
} tikh_batch_stats;

/* Build a plan for an m x n problem: sizing by Algorithm 2 (Sec. 6.2), the recursion schedule of
 * Algorithm 1 (Sec. 4.3, 6.1), transform lengths and all device workspace.  stream is a
 * cudaStream_t (NULL = legacy default stream); every later call enqueues on it.
 * Returns TIKH_EINVAL for m < 1, n < 1, unknown dtype/prec or invalid opts; TIKH_ENOMEM / TIKH_ECUDA
 * when the workspace cannot be allocated.  On failure *out is NULL. */
int tikh_plan_create(tikh_plan* out, int64_t m, int64_t n, int dtype, int prec, const tikh_opts* opts,
                     void* stream);

/* Tikhonov solution x (n entries) from device arrays col (m), row (n), b (m).  Enqueues the whole
 * path (Sec. 3-5: extension, DFT transformation, recursive basis construction, difficult points,
 * extraction x(z) = B*_1^{(j)}(z) / B*_5^{(j)}) and then synchronises the stream to report the
 * device status.  A basis longer than its planned transform (TIKH_EDEGREE) re-plans with 16x the
 * degree slack and re-runs, up to three times (tikh_stats.retries).  Returns TIKH_EINVAL for a NULL
 * pointer or an invalid lambda, TIKH_ENUMERIC / TIKH_EDIFFICULT / TIKH_ETIMEOUT when the device
 * reported a failure, TIKH_ECUDA when a launch failed.  With opts.graph the call replays its graph. */
int tikh_solve(tikh_plan plan, const void* col, const void* row, const void* b, double lambda, void* x);

/* As tikh_solve, without the final synchronisation: the status of this solve is returned by the
 * next tikh_sync.  A TIKH_EDEGREE status cannot be retried here; use tikh_solve for that. */
int tikh_solve_async(tikh_plan plan, const void* col, const void* row, const void* b, double lambda, void* x);

/* x = (T^H T + lambda I)^{-1} y for a given right-hand side y (n entries, device), the form the
 * paper's experiments solve (Sec. 7.1).  Requires m >= n (the tall, stable formulation). */
int tikh_solve_normal(tikh_plan plan, const void* col, const void* row, const void* y, double lambda, void* x);

/* Adjoint of x = (T^H T + lambda I)^{-1} T^H b for a real loss L (m >= n; TIKH_EINVAL otherwise).
 * Inputs (device, plan dtype): col, row, b, lambda as in tikh_solve, x = the solution, dLdx = dL/dx in
 * the conjugate-Wirtinger convention (dL = Re(dLdx^H dx), PyTorch's convention).  With A = T^H T +
 * lambda I and g = A^{-1} dLdx -- one more superfast solve with dLdx as its right-hand side, refined
 * like tikh_solve --:  dLdb = T g;  *dLdlambda = -Re(g^H x) (host double);  dLdcol[d] = sum_j
 * r_{j+d} conj(g_j) - u_{j+d} conj(x_j) for the diagonal a_d (d >= 0), dLdrow[d] the same for a_{-d}
 * (d >= 1), dLdrow[0] = 0, with r = b - T x and u = T g, evaluated as two FFT cross-correlations.
 * Real dtype returns real parts.  The first call allocates the adjoint workspace; synchronises. */
int tikh_solve_grad(tikh_plan plan, const void* col, const void* row, const void* b, double lambda, const void* x,
                    const void* dLdx, void* dLdcol, void* dLdrow, void* dLdb, double* dLdlambda);

/* tikh_solve_grad for `batch` problems of the plan's shape in one pass (each its own col, row, b, lambda,
 * x and dL/dx; element strides as for tikh_solve_strided, each >= the vector's length: gradients of shared
 * inputs are not summed here).  Outputs are dense: dLdcol [batch][m], dLdrow [batch][n], dLdb [batch][m]
 * (device), dLdlambda [batch] (host).  1 <= batch <= opts.batch.  Synchronises. */
int tikh_solve_grad_strided(tikh_plan plan, int batch, const void* col, int64_t col_stride, const void* row,
                            int64_t row_stride, const void* b, int64_t b_stride, const double* lambdas, const void* x,
                            int64_t x_stride, const void* dLdx, int64_t dLdx_stride, void* dLdcol, void* dLdrow,
                            void* dLdb, double* dLdlambda);

/* `batch` problems of the plan's shape in one pass: every step of the method is one launch for all of
 * them (a batch shares the recursion schedule; each problem keeps its own tau-degrees, pivots and
 * basis).  Problem i reads col + i*col_stride, row + i*row_stride, b + i*b_stride and lambdas[i]
 * (HOST array of batch doubles) and writes x + i*x_stride; strides count elements of the plan's
 * dtype, and a stride of 0 shares one array across the batch (e.g. a regularisation path: one T and
 * b, many lambdas).  1 <= batch <= opts.batch; x_stride >= n when batch > 1.  Synchronises like
 * tikh_solve; the status is the worst over the batch. */
int tikh_solve_strided(tikh_plan plan, int batch, const void* col, int64_t col_stride, const void* row,
                       int64_t row_stride, const void* b, int64_t b_stride, const double* lambdas, void* x,
                       int64_t x_stride);

/* tikh_solve with HOST arrays: copies col, row, b to the plan's device staging buffers, solves and
 * copies x back, all on the plan's stream; returns after x is in host memory. */
int tikh_solve_host(tikh_plan plan, const void* col, const void* row, const void* b, double lambda, void* x);

/* Wait for the plan's stream and return (then clear) the device status of the solves since the last
 * synchronising call: TIKH_OK, TIKH_ENUMERIC, TIKH_EDIFFICULT, TIKH_ETIMEOUT, TIKH_EDEGREE (not retried
 * here) or TIKH_ECUDA. */
int tikh_sync(tikh_plan plan);

/* Conditions the leaves deferred as difficult points (Sec. 5) in the last solve of problem 0 of the
 * call: *count = how many were deferred, ids[0 .. min(count, cap, opts.max_difficult)) = their ids
 * 2e + f (node e, omega^e; f = 0: the F condition, 1: the G condition of Eq. (interp)), in no
 * particular order.  ids is a HOST array of cap entries (NULL when cap = 0).  Synchronises the plan's
 * stream.  TIKH_EINVAL for a NULL plan or count, or cap < 0. */
int tikh_get_difficult(tikh_plan plan, int64_t* ids, int64_t cap, int64_t* count);

/* Statistics of the plan and of the last synchronised solve (*out is overwritten).  TIKH_EINVAL for a
 * NULL plan or out. */
int tikh_get_stats(tikh_plan plan, tikh_stats* out);

/* Profiling switch: flags bit 0 records a CUDA event pair around every leaf launch (Eq. (spbasis)
 * kernel) on the plan's stream; every synchronising call adds them to tikh_stats.prof_leaf_ms and
 * prof_leaf_launches.  Bit 1 records a pair around every launch group of the solve and sums them by
 * kind into prof_kind_ms / prof_kind_count.  This call resets all of them; flags = 0 turns profiling
 * off.  Profiled solves run as stream launches (no graph replay); the events add a little host and
 * device time.  TIKH_EINVAL for flags outside 0..3. */
int tikh_set_profiling(tikh_plan plan, int flags);

/* Release all device and host memory of the plan.  NULL is ignored. */
void tikh_plan_destroy(tikh_plan plan);

/* Static description of a status code. */
const char* tikh_strerror(int status);

/* ---- the Toeplitz-Gramian problem (Sec. 3.4) ---- */

/* Plan for x = (G + L^H L)^{-1} y, the Tikhonov system of min ||T x - b||^2 + ||L x||^2 when the Gramian
 * G = T^H T is an n x n Toeplitz matrix (so y = T^H b), with a p x n Toeplitz regulariser L (Sec. 3.4,
 * Eq. (gramblk), (ex7)).  The extended system has the l2 problem's two block rows and five components,
 * with L in the role of T and G's circulant extension in place of lambda I: N = 2^p M >= max(n, p) + n - 1
 * by Algorithm 2, L's extension k = N - (p + n - 1).  dtype, prec, opts and stream as for
 * tikh_plan_create (refinement residual: y - (G + L^H L) x).  TIKH_EINVAL for n < 1, p < 1 or invalid
 * options.  Such a plan serves only tikh_solve_gramian. */
int tikh_plan_create_gramian(tikh_plan* out, int64_t n, int64_t p, int dtype, int prec, const tikh_opts* opts,
                             void* stream);

/* x (n) = (G + L^H L)^{-1} y for DEVICE arrays: g = first column of the Hermitian Toeplitz G (n entries;
 * G[i][j] = g_{i-j}, g_{-d} = conj(g_d); for real data g is real and G symmetric), lcol (p) and lrow (n) =
 * first column and first row of L (lrow[0] ignored), y (n).  Synchronises like tikh_solve.  TIKH_EINVAL
 * for a NULL pointer or a plan not made by tikh_plan_create_gramian. */
int tikh_solve_gramian(tikh_plan plan, const void* g, const void* lcol, const void* lrow, const void* y, void* x);

/* ---- the general problem (Sec. 3.2) ---- */

/* Plan for min ||T x - b||^2 + ||L x||^2, i.e. x = (T^H T + L^H L)^{-1} T^H b, with T an m x n and L a pl x n
 * Toeplitz matrix (Sec. 3.2, Eq. (ex1)-(ex3)).  The extended system has three block rows, so three
 * interpolation conditions F, G, H per node (Eq. (interp)) and a 7 x 7 polynomial basis with
 * tau = [n-1, m-1, pl-1, N-n-1, N-m-1, N-pl-1, 0] (Eq. (taudef) for unequal sizes, all three block rows
 * extended to the same N); N = 2^p M >= max(m, pl) + n - 1 by Algorithm 2 with three condition sets per
 * node (a leaf holds 3 M <= opts.n_lim conditions, at most 42).  Any m, n, pl >= 1 with T^H T + L^H L
 * non-singular (m < n needs no separate form).  dtype, opts and stream as for tikh_plan_create (opts NULL:
 * n_lim 30 and eps_diff 1e-12, the measured threshold below which deferring a condition to the end stops
 * costing accuracy for this problem); the stages
 * run in FP64 (refinement residual: y - (T^H T + L^H L) x).  TIKH_EINVAL for m, n or pl < 1, invalid
 * options or a leaf size above 42 conditions.  Such a plan serves only the tikh_solve_general* calls. */
int tikh_plan_create_general(tikh_plan* out, int64_t m, int64_t n, int64_t pl, int dtype, const tikh_opts* opts,
                             void* stream);

/* x (n) = (T^H T + L^H L)^{-1} T^H b for DEVICE arrays col (m) / row (n) = first column / first row of T
 * (row[0] ignored), lcol (pl) / lrow (n) = those of L (lrow[0] ignored), b (m).  Synchronises like
 * tikh_solve.  TIKH_EINVAL for a NULL pointer or a plan not made by tikh_plan_create_general. */
int tikh_solve_general(tikh_plan plan, const void* col, const void* row, const void* lcol, const void* lrow,
                       const void* b, void* x);

/* The same with the right-hand side y (n) of the normal equations given: x = (T^H T + L^H L)^{-1} y. */
int tikh_solve_general_normal(tikh_plan plan, const void* col, const void* row, const void* lcol, const void* lrow,
                              const void* y, void* x);

/* batch (<= opts.batch) problems of the plan's shape in one call, problem i's arrays at base + i * stride
 * elements (when batch > 1: an input stride is 0, one array shared by all, or >= the array's length;
 * x_stride >= n): every launch serves all of them. */
int tikh_solve_general_strided(tikh_plan plan, int batch, const void* col, int64_t col_stride, const void* row,
                               int64_t row_stride, const void* lcol, int64_t lcol_stride, const void* lrow,
                               int64_t lrow_stride, const void* b, int64_t b_stride, void* x, int64_t x_stride);

/* Weighted Gramian of non-uniform Fourier samples (Sec. 7.4): K samples X_k = sum_s x_s exp(-2 pi i f_k s)
 * of a length-n signal at frequencies f_k in [-1/2, 1/2) with density weights w_k give the Toeplitz-Gramian
 * system (A^H W A + L^H L) x = A^H W X.  Writes its Hermitian Toeplitz Gramian's first column
 * g_d = sum_k w_k exp(+2 pi i f_k d) and the right-hand side y_s = sum_k w_k X_k exp(+2 pi i f_k s),
 * d, s = 0..n-1, by direct FP64 sums (phases reduced to [-1/2, 1/2] before sincospi).  DEVICE arrays:
 * f, w (K doubles), X (K complex128), g, y (n complex128).  Synchronises the stream.  TIKH_EINVAL for
 * K < 1, n < 1 or a NULL pointer. */
int tikh_nufft_gramian(int64_t K, const double* f, const double* w, const void* X, int64_t n, void* g, void* y,
                       void* stream);

/* ---- batches of problems of different shapes (Sec. 6.2 sizing per problem) ---- */

/* Plan for nprob problems of shapes m[i] x n[i] (HOST arrays), each solved for the same nlambda
 * regularisation weights: nprob * nlambda items (problem, lambda).  Problems whose core problems get the
 * same N = 2^p M from Algorithm 2 (Sec. 6.2) -- and the same m < n form -- form one group and share one
 * recursion schedule (each product transform as long as its longest member needs); every launch of a
 * group serves all its items at once, each with its own sizes m, n, k, tau-degrees and basis.  Groups run
 * concurrently on streams of their own, forked from and joined to `stream`.  A group whose items do not
 * fit the workspace budget runs in sequential waves: max_workspace_bytes bounds the plan's device
 * memory (0: 60 % of the free memory at creation).  opts as for tikh_plan_create (opts.batch ignored;
 * opts.graph = 1 captures the whole batch -- every wave of every group -- as one CUDA graph on the first
 * call and replays it).  TIKH_EINVAL for nprob < 1, nlambda < 1, a size < 1 or invalid options. */
int tikh_batch_plan_create(tikh_batch_plan* out, int nprob, const int64_t* m, const int64_t* n, int nlambda, int dtype,
                           int prec, const tikh_opts* opts, int64_t max_workspace_bytes, void* stream);

/* x[i * nlambda + l] = argmin ||T_i x - b_i||^2 + lambdas[l] ||x||^2 for every problem i and weight l.
 * m, n: the plan's shapes (checked); col, row, b: HOST arrays of nprob DEVICE pointers (problem i's first
 * column, first row and right-hand side, the plan's dtype); lambdas: HOST array of nlambda weights;
 * x: HOST array of nprob * nlambda DEVICE pointers to n[i] entries each.  Synchronises the plan's stream;
 * returns the worst status over all items (TIKH_EDEGREE is retried internally with more degree slack). */
int tikh_solve_batched(tikh_batch_plan plan, int nprob, const int64_t* m, const int64_t* n, const void* const* col,
                       const void* const* row, const void* const* b, int nlambda, const double* lambdas,
                       void* const* x);

/* Profiling of a batch plan: flags as for tikh_set_profiling (bit 1: every launch group timed by kind),
 * applied to every group; while it is on, calls run the groups one after another on the plan's stream
 * (no concurrency between groups, no graph), so the per-kind times do not overlap.  Resets the sums.
 * TIKH_EINVAL for a NULL plan or flags outside 0..3. */
int tikh_batch_set_profiling(tikh_batch_plan plan, int flags);

/* Statistics of the batch plan and its last call.  TIKH_EINVAL for a NULL plan or out. */
int tikh_batch_get_stats(tikh_batch_plan plan, tikh_batch_stats* out);

/* Release the batch plan's streams, graphs and device memory.  NULL is ignored. */
void tikh_batch_plan_destroy(tikh_batch_plan plan);

/* ---- test hooks: one building block on caller data (device pointers), for stage-wise parity ---- */

/* In-place DFT of n complex128 values (device): X_k = sum_j x_j exp(sign 2 pi i jk / n), sign = +1
 * evaluates the coefficient vector at the n-th roots of unity (Sec. 4.1, Eq. (vandprod)); unnormalised.
 * n must factor into 2, 3, 5, 7 and be at most 4096^2.  Synchronises the stream; TIKH_EINVAL otherwise. */
int tikh_test_fft(int64_t n, void* data, int sign, void* stream);

/* tikh_test_fft in FP32: n complex64 values (interleaved float re, im) transformed in place by the same
 * engine instantiated for complex64 (FP32 butterflies and twiddles rounded from the FP64 tables), as used
 * by the recursion's FFT stages under TIKH_PREC_FP32 / TIKH_PREC_FP32_REFINE. */
int tikh_test_fft32(int64_t n, void* data, int sign, void* stream);

/* The leaf's reciprocal of a pivot magnitude on n positive normal doubles (device arrays d, out; biased
 * exponent of each d in (2, 2044)): an FP32 approximate-reciprocal seed of d's 23 leading mantissa bits
 * refined by one third-order step of the series 1/d = y0 (1 + e + e^2 + ...), e = 1 - d y0, which is
 * within FP64 rounding of 1/d.  Synchronises the stream.  TIKH_EINVAL for n < 1 or a NULL pointer. */
int tikh_test_rcp(int64_t n, const double* d, double* out, void* stream);

/* The power-of-two column scaling of the basis (the bases of Sec. 4.3 carried with lazy column scales): for
 * each i, v[i] times the scale of the column maximum bits[i] (the bit pattern of a non-negative double; the
 * scale 2^k puts that maximum in [0.5, 1)), once by an add to the exponent field (out_exp, what the
 * products' loaders use) and once by an FP64 multiply (out_mul).  The two agree bit for bit.  Device
 * arrays; synchronises the stream.  TIKH_EINVAL for n < 1 or a NULL pointer. */
int tikh_test_scale(int64_t n, const double* v, const unsigned long long* bits, double* out_exp, double* out_mul,
                    void* stream);

/* One leaf of Algorithm 1: the serial single-point construction of Eq. (spbasis) (Sec. 4.3) with
 * condition pivoting and difficult-point deferral (Sec. 5) over K <= 64 conditions.
 * Inputs (device): sigma (K complex128 nodes), r (K x 5 complex128 residual rows), delta_in (5 ints,
 * starting tau-degrees), eps (deferral threshold).  Outputs (device): B (25 entries x (K+1) complex128,
 * entry (i,j) at (5i+j)(K+1), unscaled), len (25 ints, trimmed to the degree bounds), delta_out (5 ints),
 * order / pivot (K ints: position and pivot column processed at each step, -1 after the last),
 * deferred (K int64 positions, unordered) and n_def (1 int).  Synchronises the stream. */
int tikh_test_leaf(int K, const void* sigma, const void* r, const int* delta_in, double eps, void* B, int* len,
                   int* delta_out, int* order, int* pivot, int64_t* deferred, int* n_def, void* stream);

/* Measured peak FMA rate of the current device (the roofline denominator of FP64- and FP32-bound
 * kernels): kind 0 = FP64 (DFMA), 1 = FP32 (FFMA).  A kernel of 4 CTAs x 256 threads per SM, each thread
 * running 8 independent FMA chains with no memory traffic, timed with CUDA events on `stream` (best of
 * three after a warm-up launch).  *gflops = 2 x FMAs / seconds / 1e9.  Synchronises the stream.
 * TIKH_EINVAL for a NULL gflops or another kind. */
int tikh_test_peak(int kind, double* gflops, void* stream);

/* ---- one solver for many right-hand sides ---- */

/* The paper's solver builds one interpolation basis per right-hand side: b enters the conditions' fifth
 * component and every pivot decision (Sec. 4.3).  For many right-hand sides of one T and lambda this
 * extension (the paper has none) reuses the matrix instead: A = T^H T + lambda I has displacement rank 4
 * (A - Z A Z^H, Z the down-shift), and so has X = A^{-1}.  Eight superfast solves X v_i (right-hand sides
 * built from T's first row, first column, last column and A e_0) give four pairs (u_t, w_t) with
 *   X = sum_t H(u_t) H(w_t)^H,   H(u)_{ik} = u_{i+k} (0 for i + k >= n)  (Hankel),
 * and every further right-hand side costs ten length-N transforms (twelve from b), plus fourteen per
 * refinement correction x += X~(y - A x) (the residual by the FFT matvec of Sec. 7.3, as in Sec. 7.2).
 * The handle keeps the spectra of the four pairs and of T's generator (9 N complex128) and the workspace
 * of one pass over up to max_rhs right-hand sides (about 13 max_rhs N complex128). */
typedef struct tikh_inverse_s* tikh_inverse;

/* Build the representation for the l2 plan `plan` (m >= n; not a Toeplitz-Gramian or general plan) with
 * T given by col, row (device arrays of the plan's dtype) and weight lambda > 0.  The eight solves run on
 * the plan (its options apply: batch size, refinement, graph) in batches of opts.batch; the plan must
 * outlive the handle and must not run other calls concurrently with it (same stream).  max_rhs in
 * 1..4096.  Synchronises; returns the first failing solve's status, TIKH_ENOMEM, or TIKH_EINVAL. */
int tikh_inverse_create(tikh_inverse* out, tikh_plan plan, const void* col, const void* row, double lambda,
                        int max_rhs);

/* x_r = (T^H T + lambda I)^{-1} T^H b_r (normal = 0; b_r has m entries) or (T^H T + lambda I)^{-1} y_r
 * (normal = 1; n entries), r < nrhs, then refine_steps (0..16) corrections each.  Right-hand side r at
 * b + r * b_stride, its solution at x + r * x_stride (device arrays, plan dtype; strides in elements,
 * >= the vector lengths when nrhs > 1).  Passes of max_rhs right-hand sides.  Synchronises. */
int tikh_inverse_apply(tikh_inverse inv, int nrhs, const void* b, int64_t b_stride, void* x, int64_t x_stride,
                       int normal, int refine_steps);

/* Copy u_0..u_3, w_0..w_3 (8 n complex128, n apart) to the device array out.  Synchronises. */
int tikh_inverse_generators(tikh_inverse inv, void* out);

/* Kernels launched by the last create or apply, and the handle's device bytes. */
int tikh_inverse_info(tikh_inverse inv, int64_t* kernel_launches, int64_t* workspace_bytes);

void tikh_inverse_destroy(tikh_inverse inv);

/* ---- allocation-free variant ---- */

/* The DFT of tikh_test_fft (same transform, same kernels, same result) for callers that must not
 * allocate device memory during the call: code whose device memory is owned by another allocator or
 * a fixed budget (a cudaMalloc there would take memory the caller has promised elsewhere, or fail),
 * and latency-critical loops that cannot afford an allocation and the synchronisation it implies.
 * The paper has no counterpart; this is an interface convenience.
 * Its scratch (twiddle tables and the four-step temporary, about 2.2 MB) is one file-scope device
 * array that every GPU loading the library keeps until process exit; nothing is allocated or freed
 * per call (no cudaMalloc, cudaFree or allocating library routine).
 * n must factor into 2, 3, 5, 7 and be at most 65536 (larger n returns TIKH_EINVAL: use
 * tikh_test_fft).  data: n complex128 values on the device, transformed in place; the call
 * synchronises the stream.
 * The first call on each device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current.  Every call rewrites the
 * parts of the scratch it reads, so nothing needs clearing, but all calls share the one array: calls
 * that overlap on the GPU (other streams, other host threads) race and must be serialised by the
 * caller. */
int tikh_fft_noalloc(int64_t n, void* data, int sign, void* stream);

#ifdef __cplusplus
}
#endif
#endif
