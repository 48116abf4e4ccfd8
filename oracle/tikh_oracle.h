/*
 * tikh_oracle.h -- plain CPU FP64 oracle for the l2-penalised superfast Tikhonov solver of
 * Turnes, Balcan & Romberg, "Superfast Tikhonov Regularization of Toeplitz Systems" (arXiv 1302.6945).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this code: only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg do.  It shares no code, header,
 * table or helper with the CUDA library.  It is slow on purpose: every step is the plain
 * definition or the paper's algorithm in the paper's order.
 *
 * Conventions shared by every function:
 *  - complex arrays are interleaved (re, im) doubles;
 *  - T is m x n Toeplitz, T[i][j] = a_{i-j}; col[d] = a_d (d = 0..m-1), row[d] = a_{-d}
 *    (d = 1..n-1; row[0] is ignored);
 *  - nodes are omega_e = exp(+2 pi i e / N) (Sec. 4.1, Eq. (vandprod));
 *  - basis polynomials are stored lowest coefficient first.
 * Return value 0 = success; negative = error (see TIKH_ORACLE_E*).
 */
#ifndef TIKH_ORACLE_H
#define TIKH_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define TIKH_ORACLE_OK 0
#define TIKH_ORACLE_EINVAL (-1)
#define TIKH_ORACLE_ENOMEM (-2)
#define TIKH_ORACLE_ENUMERIC (-3) /* final degree pattern is not one 0 and four 1s */

/* evaluation / product modes for the recursive steps 2 and 4 of Algorithm 1 */
#define TIKH_ORACLE_AUTO 0   /* direct for small nodes, FFT for large */
#define TIKH_ORACLE_DIRECT 1 /* Horner evaluation and schoolbook products only */
#define TIKH_ORACLE_FFT 2    /* FFT evaluation and FFT products only */

typedef struct {
  int nlim;         /* leaf cutoff N_lim (Sec. 6.2); leaves hold <= 2*M conditions */
  int m_min;        /* lower bound on M (forces a larger extension k); 0 = none */
  double eps_diff;  /* difficult-point threshold on |r_pivot|/||r||_2 (Sec. 5) */
  int mode;         /* TIKH_ORACLE_AUTO / DIRECT / FFT */
  int fill;         /* arbitrary extension entries: 0 = seeded pseudo-random of the coefficients' size,
                       1 = linear ramp between a_{m-1} and a_{-(n-1)} */
  int is_complex;   /* 1: complex data (complex fill values); 0: real data (real fill values) */
} tikh_oracle_opts;

typedef struct {
  int64_t N, M, k; /* nodes, leaf size parameter, extension size */
  int p;           /* number of paired-interleaving splits */
  int64_t n_difficult; /* conditions deferred to the end (Sec. 5, difficult points) */
  int64_t n_dropped;   /* conditions whose residual was exactly zero (already satisfied) */
  int delta[7];        /* final tau-degrees of the basis columns (5 used by the l2 and Gramian solves) */
  int jstar;           /* the column with tau-degree 0 */
  int dual;            /* 1 when m < n was solved through T^H (T T^H + lam I)^{-1} b */
} tikh_oracle_stats;

/* Algorithm 2 (OptExtend) for the l2 case: two condition sets, paired interleaving, M even and
 * 7-smooth (so every FFT length has factors 2, 3, 5, 7 only).  Outputs N = 2^p M, k = N - (m+n-1). */
int tikh_oracle_plan(int64_t m, int64_t n, const tikh_oracle_opts* opts, int64_t* N, int64_t* M,
                     int64_t* k, int* p);

/* unnormalised DFT  X_k = sum_j x_j exp(sign * 2 pi i j k / n)  (textbook mixed radix). */
int tikh_oracle_fft(int64_t n, double* data, int sign);

/* Interpolation conditions F_k, G_k (k = 0..N-1, each 5 complex) of the l2 system (Eq. (ex6),
 * Sec. 4.1) for the right-hand side  y = T^H b  given directly:  (T^H T + lam I) x = y.
 * F, G: N*5 complex each.  tau: 5 ints.  Requires the plan's N (call tikh_oracle_plan). */
int tikh_oracle_conditions(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                           double lam, const tikh_oracle_opts* opts, double* F, double* G, int* tau);

/* One leaf: serial single-point construction (Eq. (spbasis), Sec. 4.3) with condition pivoting
 * and difficult-point deferral, on K conditions with nodes sigma (K complex), residual rows
 * r (K*5 complex, overwritten), starting degrees delta (5 ints, updated).  Outputs the leaf basis
 * B (25 entries x cap coefficients, entry (i,j) at (5i+j)*cap), len (25 ints), the processing
 * order (K ints: position processed at each step, -1 after the last), the pivot column of each
 * step (K ints), and the deferred positions (K ints, count in *n_def).  No column scaling. */
int tikh_oracle_leaf(int K, const double* sigma, double* r, int* delta, double eps, int64_t cap,
                     double* B, int64_t* len, int* order, int* pivot, int* deferred, int* n_def);

/* Solve (T^H T + lam I) x = y through the superfast algorithm (m >= n is the stable case).
 * x: n complex.  If B is non-null, the final basis is written (25 entries x cap coefficients) with
 * lengths in len.  stats may be null. */
int tikh_oracle_solve_normal(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                             double lam, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats,
                             double* B, int64_t cap, int64_t* len);

/* tikh_oracle_solve_normal that also writes the ids 2e + f (node e, f = 0: F, 1: G) of the conditions
 * the leaves deferred as difficult (Sec. 5), in the order they were deferred, to deferred_out (at most
 * deferred_cap of them; stats->n_difficult is the full count). */
int tikh_oracle_solve_normal_ex(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                                double lam, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats,
                                double* B, int64_t cap, int64_t* len, int64_t* deferred_out, int64_t deferred_cap);

/* The Toeplitz-Gramian problem (Sec. 3.4, Eq. (gramblk), (ex7)): x = (G + L^H L)^{-1} y with G an n x n
 * Hermitian Toeplitz matrix (a Gramian T^H T that is Toeplitz) given by its first column g (n complex;
 * G[i][j] = g_{i-j}, g_{-d} = conj(g_d)) and L a pl x n Toeplitz regulariser given by its first column
 * lcol (pl) and first row lrow (n; lrow[0] ignored).  Same algorithm as the l2 solve with L in place of T
 * and G in place of lam I; N = 2^p M >= max(n, pl) + n - 1.  x: n complex. */
int tikh_oracle_solve_gramian(int64_t n, int64_t pl, const double* g, const double* lcol, const double* lrow,
                              const double* y, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats);

/* The general problem (Sec. 3.2, Eq. (ex1)-(ex3)): x = (T^H T + L^H L)^{-1} y with T an m x n and L a p x n
 * Toeplitz matrix (first columns col, lcol; first rows row, lrow, whose [0] entries are ignored).  Three
 * condition sets F, G, H per node (Eq. (interp)), a 7 x 7 basis, tau = [n-1, m-1, p-1, N-n-1, N-m-1,
 * N-p-1, 0] (Eq. (taudef) for unequal sizes); N = 2^p' M >= max(m, p) + n - 1 by Algorithm 2 with three
 * sets per node.  x: n complex. */
int tikh_oracle_plan_general(int64_t m, int64_t n, int64_t p, const tikh_oracle_opts* opts, int64_t* N,
                             int64_t* M, int* pp);
int tikh_oracle_solve_general(int64_t m, int64_t n, int64_t p, const double* col, const double* row,
                              const double* lcol, const double* lrow, const double* y, const tikh_oracle_opts* opts,
                              double* x, tikh_oracle_stats* stats);
/* The general problem's conditions: cond[N][3][7] complex (rows F, G, H of node e), tau: 7 ints. */
int tikh_oracle_conditions_general(int64_t m, int64_t n, int64_t p, const double* col, const double* row,
                                   const double* lcol, const double* lrow, const double* y,
                                   const tikh_oracle_opts* opts, double* cond, int* tau);

/* Tikhonov solution x = argmin ||T x - b||^2 + lam ||x||^2  (Eq. (tik), (tiksol)).
 * m >= n: y = T^H b then solve_normal.  m < n: x = T^H v with (T T^H + lam I) v = b, solved by the
 * same algorithm on the tall matrix T^H.  b: m complex; x: n complex. */
int tikh_oracle_solve(int64_t m, int64_t n, const double* col, const double* row, const double* b,
                      double lam, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats);

/* tikh_oracle_solve followed by `steps` iterative-refinement corrections on the core (tall) system
 * A v = y, A = T_c^H T_c + lam I: v <- v + A^{-1} (y - A v), each correction by the same superfast
 * solve.  rel_residual (may be null) receives ||y - A v|| / ||y|| after the last correction. */
int tikh_oracle_solve_refined(int64_t m, int64_t n, const double* col, const double* row, const double* b,
                              double lam, const tikh_oracle_opts* opts, int steps, double* x, tikh_oracle_stats* stats,
                              double* rel_residual);

/* y = T^H v (v: m complex, y: n complex) and u = T x (x: n, u: m), by a zero-padded circulant
 * embedding (the DFT diagonalises circulants, Eq. (circdiag)). */
int tikh_oracle_apply_th(int64_t m, int64_t n, const double* col, const double* row, const double* v, double* y);
int tikh_oracle_apply_t(int64_t m, int64_t n, const double* col, const double* row, const double* x, double* u);

#ifdef __cplusplus
}
#endif
#endif
