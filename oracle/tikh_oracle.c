/*
 * tikh_oracle.c -- plain CPU FP64 oracle for the superfast Tikhonov solver of Turnes, Balcan & Romberg
 * (arXiv 1302.6945): the l2-penalised problem, the Toeplitz-Gramian problem and the general problem.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's CPU baseline,
 * never by the product path.  It shares nothing with the CUDA library.
 *
 * Each function cites the passage it follows.  Where the paper is silent or garbled, the reading
 * taken is stated at the point of use:
 *  R1 pivot column = the column of minimum current tau-degree among the non-zero residual entries
 *     (Sec. 4.3: "the column with lowest tau-degree has its degree increased"); ties: larger
 *     |r|^2, then lower index.
 *  R2 the extension's top-left entry is a_{-(n+k-1)} (Sec. 3.1 prints a_{-n-k}): the circulant
 *     generator is c_T[j] = a_{j-(n+k-1)} over a periodic sequence of length N.
 *  R3 tau for k != 1: gamma_1 has m+k-1 and gamma_2 has n+k-1 coefficients, so
 *     tau = [n-1, m-1, m+k-2, n+k-2, 0] (Eq. (taudef) is printed for k = 1, p = 7).
 *  R4 Algorithm 1 carries the absolute tau-degrees delta: the left child starts from delta_in,
 *     the right child from the left child's output (Theorem 1 with tau_{kappa->K} = -delta).
 *  R5 the k arbitrary entries (Sec. 6.2, "similar in value") are pseudo-random with the size of
 *     the known coefficients: a = peak * u, peak = max over known d of max(|Re a_d|, |Im a_d|),
 *     u uniform in [-1, 1) from the SplitMix64 generator (Steele, Lea, Flood 2014) used as a
 *     counter-based hash of the entry index (real u for real data, u + i u' for complex).  Zero-like
 *     fills (including a linear ramp between two near-zero PSF tails) lose accuracy for large k.
 *     The T^H extension uses the same periodic sequence.  fill = 1 selects the linear ramp.
 *  R6 Algorithm 2 for two condition sets with paired interleaving: halve M while 2M > N_lim,
 *     then round M up to even (Sec. 6.2) and further to a 7-smooth number (FFT lengths with
 *     factors 2, 3, 5, 7 only; the solution does not depend on k).
 *  R7 difficult point: the best remaining condition of a leaf has |r_pi| < eps ||r||_2; it and
 *     the rest of the leaf are deferred and processed serially against the final basis.
 *  R8 condition pivoting: the next condition of a leaf is the one with the largest
 *     |r_pi|^2 / ||r||_2^2 (ties: lowest position).
 *  R9 every basis returned by a recursion node has each column scaled by a power of two so that
 *     its largest |Re|, |Im| coefficient lies in [0.5, 1); the solution is unchanged.
 *  R10 entry (i,j) of a node's basis has degree <= delta_out_j - delta_in_i; a column that was
 *     never a pivot only accumulates multiples of pivot columns, so its entries are also bounded
 *     by (largest delta_out of a pivoted column) - delta_in_i (diagonal: >= 0).  Products are
 *     trimmed to these bounds (what is cut is round-off).
 *  R11 m < n is solved as x = T^H (T T^H + lam I)^{-1} b with the same algorithm on T^H, whose
 *     right-hand-side term is b itself (Sec. 7.1 solves (G_T + G_L) x = y with y given).
 *  R22 general problem (Sec. 3.2): the three block rows of Eq. (ex3) are printed with q+n, m+n and p+n
 *     rows; the interpolation needs one node set, so all three are extended to the same N >= q + n - 1
 *     (q = max(m, p)) with N - n, N - m and N - p extension rows, and tau_i + 1 is the length of each
 *     unknown: tau = [n-1, m-1, p-1, N-n-1, N-m-1, N-p-1, 0] (Eq. (taudef) is printed for m = p = q and
 *     a 1-circulant extension).  L's arbitrary entries use SplitMix64 counters offset by 2^41.
 */
#include "tikh_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------ */
/* DFT by textbook mixed-radix decimation in time; any length (direct DFT for a large prime).  */
/* ------------------------------------------------------------------------------------------ */

static int64_t smallest_factor(int64_t n) {
  for (int64_t f = 2; f * f <= n; ++f)
    if (n % f == 0) return f;
  return n;
}

/* a[0..n): in-place DFT with twiddles tw[t] = exp(sign 2 pi i t / ntop), n | ntop */
static int fft_rec(cx* a, int64_t n, const cx* tw, int64_t ntop) {
  if (n == 1) return 0;
  int64_t r = smallest_factor(n), m = n / r, step = ntop / n;
  cx* tmp = (cx*)malloc(sizeof(cx) * (size_t)n);
  if (!tmp) return TIKH_ORACLE_ENOMEM;
  for (int64_t t = 0; t < r; ++t)
    for (int64_t j = 0; j < m; ++j) tmp[t * m + j] = a[j * r + t];
  for (int64_t t = 0; t < r; ++t) {
    int rc = fft_rec(tmp + t * m, m, tw, ntop);
    if (rc) { free(tmp); return rc; }
  }
  /* a[k1 + m k2] = sum_t w_n^{t (k1 + m k2)} sub_t[k1] */
  for (int64_t k1 = 0; k1 < m; ++k1)
    for (int64_t k2 = 0; k2 < r; ++k2) {
      int64_t kk = k1 + m * k2;
      cx s = 0;
      for (int64_t t = 0; t < r; ++t) s += tw[((t * kk) % n) * step] * tmp[t * m + k1];
      a[kk] = s;
    }
  free(tmp);
  return 0;
}

static int dft(cx* a, int64_t n, int sign) {
  if (n <= 0) return TIKH_ORACLE_EINVAL;
  cx* tw = (cx*)malloc(sizeof(cx) * (size_t)n);
  if (!tw) return TIKH_ORACLE_ENOMEM;
  for (int64_t t = 0; t < n; ++t) {
    double ang = 2.0 * M_PI * (double)t / (double)n;
    tw[t] = cos(ang) + (sign > 0 ? 1.0 : -1.0) * sin(ang) * I;
  }
  int rc = fft_rec(a, n, tw, n);
  free(tw);
  return rc;
}

int tikh_oracle_fft(int64_t n, double* data, int sign) { return dft((cx*)data, n, sign); }

/* ------------------------------------------------------------------------------------------ */
/* Plan: Algorithm 2 (OptExtend), reading R6.                                                  */
/* ------------------------------------------------------------------------------------------ */

static int is_5smooth(int64_t v) {
  while (v % 2 == 0) v /= 2;
  while (v % 3 == 0) v /= 3;
  while (v % 5 == 0) v /= 5;
  return v == 1;
}

static int is_7smooth(int64_t v) {
  while (v % 7 == 0) v /= 7;
  return is_5smooth(v);
}

/* Algorithm 2 for ns condition sets per node over a circulant of at least Nt points: halve M while
 * ns M > N_lim, then M even and 7-smooth (R6); N = 2^p M. */
static int plan_sets(int64_t Nt, int ns, const tikh_oracle_opts* opts, int64_t* N, int64_t* M, int* p) {
  if (Nt < 1 || !opts || opts->nlim < ns) return TIKH_ORACLE_EINVAL;
  int64_t Mv = Nt;
  int pv = 0;
  while (ns * Mv > opts->nlim) {
    ++pv;
    Mv = (Mv + 1) / 2;
  }
  if (Mv % 2) ++Mv;
  if (Mv < opts->m_min) Mv = opts->m_min + (opts->m_min % 2);
  while (!is_7smooth(Mv)) Mv += 2;
  *N = Mv << pv;
  *M = Mv;
  *p = pv;
  return 0;
}

int tikh_oracle_plan(int64_t m, int64_t n, const tikh_oracle_opts* opts, int64_t* N, int64_t* M, int64_t* k,
                     int* p) {
  if (m < 1 || n < 1 || !opts || opts->nlim < 2) return TIKH_ORACLE_EINVAL;
  int rc = plan_sets(m + n - 1, 2, opts, N, M, p); /* two condition sets per node: s*M with s = 2 */
  if (rc) return rc;
  *k = *N - (m + n - 1);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Toeplitz generator and the l2 interpolation conditions (Sec. 3.1, 3.3, 4.1).                */
/* ------------------------------------------------------------------------------------------ */

/* SplitMix64 output for counter value c (Steele, Lea, Flood 2014), mapped to [-1, 1) */
static double splitmix_uniform(uint64_t c) {
  uint64_t z = 0x5eedULL + (c + 1) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* periodic sequence at[d mod N] = a_d on d in [-(n-1), m-1]; k arbitrary entries filled by R5 (SplitMix64
 * counters from ctr0: 0 for T, 2^41 for a general regulariser L) */
static void periodic_generator(int64_t m, int64_t n, int64_t N, int64_t k, const cx* col, const cx* row,
                               int fill, int is_complex, uint64_t ctr0, cx* at) {
  for (int64_t d = 0; d < N; ++d) at[d] = 0;
  for (int64_t d = 0; d < m; ++d) at[d % N] = col[d];
  for (int64_t d = 1; d < n; ++d) at[(N - d) % N] = row[d];
  if (fill == 1) {
    cx lo = (n > 1) ? row[n - 1] : col[0]; /* a_{-(n-1)} */
    cx hi = col[m - 1];                    /* a_{m-1} */
    for (int64_t i = 1; i <= k; ++i) at[(m - 1 + i) % N] = hi + (lo - hi) * ((double)i / (double)(k + 1));
    return;
  }
  double peak = 0.0;
  for (int64_t d = 0; d < m; ++d) {
    if (fabs(creal(col[d])) > peak) peak = fabs(creal(col[d]));
    if (fabs(cimag(col[d])) > peak) peak = fabs(cimag(col[d]));
  }
  for (int64_t d = 1; d < n; ++d) {
    if (fabs(creal(row[d])) > peak) peak = fabs(creal(row[d]));
    if (fabs(cimag(row[d])) > peak) peak = fabs(cimag(row[d]));
  }
  for (int64_t i = 1; i <= k; ++i) {
    double re = peak * splitmix_uniform((uint64_t)(2 * i) + ctr0);
    double im = is_complex ? peak * splitmix_uniform((uint64_t)(2 * i + 1) + ctr0) : 0.0;
    at[(m - 1 + i) % N] = re + im * I;
  }
}

/* unit-modulus node omega^e for e taken mod N */
static cx node(int64_t e, int64_t N) {
  e %= N;
  if (e < 0) e += N;
  double ang = 2.0 * M_PI * (double)e / (double)N;
  return cos(ang) + sin(ang) * I;
}

/* F, G per Sec. 4.1 specialised to the reduced l2 system (Eq. (ex6)), right-hand side y:
 *   block row 1 (m+k-1 extension rows, then n rows):  lam*x + T^H sigma_1 + gamma_1 - y = 0
 *   block row 2 (n+k-1 extension rows, then m rows): -T x + sigma_1 + gamma_2 = 0
 * unknowns p = [x (n), sigma_1 (m), gamma_1 (m+k-1), gamma_2 (n+k-1), 1]; left-multiplying each
 * block row by the DFT turns each partial circulant into the DFT of its generator (Eq. (circdiag)).
 */
static int build_conditions(int64_t m, int64_t n, int64_t N, int64_t k, const cx* col, const cx* row, const cx* y,
                            double lam, int fill, int is_complex, cx* F, cx* G) {
  cx* at = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cT = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cH = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cy = (cx*)malloc(sizeof(cx) * (size_t)N);
  int rc = TIKH_ORACLE_ENOMEM;
  if (!at || !cT || !cH || !cy) goto done;
  periodic_generator(m, n, N, k, col, row, fill, is_complex, 0, at);
  for (int64_t j = 0; j < N; ++j) {
    int64_t dT = ((j - (n + k - 1)) % N + N) % N; /* c_T[j]  = a_{j-(n+k-1)}         (R2) */
    int64_t dH = ((m + k - 1 - j) % N + N) % N;   /* c_H[j]  = conj(a_{(m+k-1)-j})   (T^H) */
    cT[j] = at[dT];
    cH[j] = conj(at[dH]);
    cy[j] = 0;
  }
  /* generator of the column of the constant unknown: -y placed after the m+k-1 extension rows */
  for (int64_t i = 0; i < n; ++i) cy[m + k - 1 + i] = -y[i];
  if ((rc = dft(cT, N, +1)) || (rc = dft(cH, N, +1)) || (rc = dft(cy, N, +1))) goto done;
  for (int64_t e = 0; e < N; ++e) {
    cx* f = F + 5 * e;
    cx* g = G + 5 * e;
    f[0] = lam * node(e * (m + k - 1), N); /* lam I_n below m+k-1 zero rows: generator lam e_{m+k-1} */
    f[1] = cH[e];                          /* circulant extension of T^H */
    f[2] = 1.0;                            /* [I_{m+k-1}; 0]: generator e_0 */
    f[3] = 0.0;
    f[4] = cy[e];
    g[0] = -cT[e];                   /* -C_k(T) */
    g[1] = node(e * (n + k - 1), N); /* [0; I_m] below n+k-1 rows: generator e_{n+k-1} */
    g[2] = 0.0;
    g[3] = 1.0; /* [I_{n+k-1}; 0] */
    g[4] = 0.0;
  }
  rc = 0;
done:
  free(at); free(cT); free(cH); free(cy);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Polynomial w x w matrices (w = 5 for the l2 and Toeplitz-Gramian systems, 7 for the general   */
/* problem of Sec. 3.2).                                                                      */
/* ------------------------------------------------------------------------------------------ */

#define WMAX 7

typedef struct {
  int w;                 /* matrix size */
  cx* c[WMAX * WMAX];    /* entry (i, j) at c[w i + j] */
  int64_t len[WMAX * WMAX]; /* number of stored coefficients; 0 = the zero polynomial */
} pmat;

static void pm_free(pmat* B) {
  for (int e = 0; e < WMAX * WMAX; ++e) { free(B->c[e]); B->c[e] = NULL; B->len[e] = 0; }
}

static int pm_identity(pmat* B, int w) {
  memset(B, 0, sizeof(*B));
  B->w = w;
  for (int i = 0; i < w; ++i) {
    B->c[(w + 1) * i] = (cx*)malloc(sizeof(cx));
    if (!B->c[(w + 1) * i]) return TIKH_ORACLE_ENOMEM;
    B->c[(w + 1) * i][0] = 1.0;
    B->len[(w + 1) * i] = 1;
  }
  return 0;
}

/* ensure entry e can hold len coefficients (new ones zero) */
static int pm_reserve(pmat* B, int e, int64_t len) {
  if (B->len[e] >= len) return 0;
  cx* nc = (cx*)realloc(B->c[e], sizeof(cx) * (size_t)len);
  if (!nc) return TIKH_ORACLE_ENOMEM;
  for (int64_t t = B->len[e]; t < len; ++t) nc[t] = 0;
  B->c[e] = nc;
  B->len[e] = len;
  return 0;
}

static cx horner(const cx* c, int64_t len, cx z) {
  cx v = 0;
  for (int64_t t = len - 1; t >= 0; --t) v = v * z + c[t];
  return v;
}

/* ------------------------------------------------------------------------------------------ */
/* Serial single-point construction (Eq. (spbasis), Sec. 4.3) with pivoting (R1, R7, R8).       */
/* ------------------------------------------------------------------------------------------ */

/* Processes the conditions (sigma[q], r[q]) q < K (rows of B->w entries) against basis B (updated in place,
 * B <- B E_q).  active[q] != 0 marks the conditions still to process.  eps < 0 disables deferral.
 * order/pivot (may be null) record the processing; deferred (may be null) collects deferred
 * positions; n_drop counts conditions whose residual is exactly zero. */
static int serial_construct(int K, const cx* sigma, cx* r, char* active, int* delta, double eps, pmat* B,
                            int* order, int* pivot, int* deferred, int* n_def, int64_t* n_drop) {
  const int w = B->w;
  int step = 0;
  if (n_def) *n_def = 0;
  for (;;) {
    int best = -1, bpi = -1;
    double bscore = -1.0;
    for (int q = 0; q < K; ++q) {
      if (!active[q]) continue;
      const cx* rq = r + w * q;
      double mag[WMAX], tot = 0.0;
      int pi = -1;
      for (int i = 0; i < w; ++i) {
        mag[i] = creal(rq[i]) * creal(rq[i]) + cimag(rq[i]) * cimag(rq[i]);
        tot += mag[i];
      }
      for (int i = 0; i < w; ++i) {
        if (creal(rq[i]) == 0.0 && cimag(rq[i]) == 0.0) continue; /* R1: non-zero entries only */
        if (pi < 0 || delta[i] < delta[pi] || (delta[i] == delta[pi] && mag[i] > mag[pi])) pi = i;
      }
      if (pi < 0) { /* exactly zero residual: the condition is already satisfied */
        active[q] = 0;
        if (n_drop) ++*n_drop;
        continue;
      }
      double score = mag[pi] / tot; /* R8 */
      if (score > bscore) { bscore = score; best = q; bpi = pi; }
    }
    if (best < 0) break;
    if (eps >= 0.0 && bscore < eps * eps) { /* R7: defer this and every remaining condition */
      for (int q = 0; q < K; ++q)
        if (active[q]) {
          active[q] = 0;
          if (deferred) deferred[(*n_def)++] = q;
        }
      break;
    }
    const int pi = bpi;
    const cx sg = sigma[best];
    const cx* rs = r + w * best;
    /* mu_i = -r_i / r_pi, division as r_i * conj(r_pi) / |r_pi|^2 */
    double den = creal(rs[pi]) * creal(rs[pi]) + cimag(rs[pi]) * cimag(rs[pi]);
    cx inv = creal(rs[pi]) / den - (cimag(rs[pi]) / den) * I;
    cx mu[WMAX];
    for (int i = 0; i < w; ++i) mu[i] = (i == pi) ? 0.0 : -(rs[i] * inv);
    active[best] = 0;
    if (order) order[step] = best;
    if (pivot) pivot[step] = pi;
    ++step;
    /* residual update r_q <- r_q E(sigma_q): E = I except column pi = (z - sg) e_pi + sum mu_i e_i */
    for (int q = 0; q < K; ++q) {
      if (!active[q]) continue;
      cx* rq = r + w * q;
      cx rp = rq[pi];
      for (int i = 0; i < w; ++i)
        if (i != pi) rq[i] = rq[i] + mu[i] * rp;
      rq[pi] = rp * (sigma[q] - sg);
    }
    /* basis update B <- B E: column pi <- (z - sg) column pi; column i += mu_i * old column pi */
    for (int row = 0; row < w; ++row) {
      int ep = w * row + pi;
      int64_t L = B->len[ep];
      if (L == 0) continue;
      cx* old = (cx*)malloc(sizeof(cx) * (size_t)L);
      if (!old) return TIKH_ORACLE_ENOMEM;
      memcpy(old, B->c[ep], sizeof(cx) * (size_t)L);
      for (int i = 0; i < w; ++i) {
        if (i == pi) continue;
        int ei = w * row + i;
        if (pm_reserve(B, ei, L)) { free(old); return TIKH_ORACLE_ENOMEM; }
        for (int64_t t = 0; t < L; ++t) B->c[ei][t] = B->c[ei][t] + mu[i] * old[t];
      }
      if (pm_reserve(B, ep, L + 1)) { free(old); return TIKH_ORACLE_ENOMEM; }
      B->c[ep][0] = -(sg * old[0]);
      for (int64_t t = 1; t < L; ++t) B->c[ep][t] = old[t - 1] - sg * old[t];
      B->c[ep][L] = old[L - 1];
      free(old);
    }
    delta[pi] += 1;
  }
  if (order)
    for (int s = step; s < K; ++s) order[s] = -1;
  if (pivot)
    for (int s = step; s < K; ++s) pivot[s] = -1;
  return 0;
}

int tikh_oracle_leaf(int K, const double* sigma, double* r, int* delta, double eps, int64_t cap, double* B,
                     int64_t* len, int* order, int* pivot, int* deferred, int* n_def) {
  if (K < 0 || !sigma || !r || !delta || !B || !len) return TIKH_ORACLE_EINVAL;
  pmat P;
  int rc = pm_identity(&P, 5);
  char* active = (char*)malloc((size_t)K + 1);
  if (rc || !active) { pm_free(&P); free(active); return TIKH_ORACLE_ENOMEM; }
  memset(active, 1, (size_t)K);
  int64_t ndrop = 0;
  int nd = 0;
  rc = serial_construct(K, (const cx*)sigma, (cx*)r, active, delta, eps, &P, order, pivot, deferred, &nd, &ndrop);
  if (!rc) {
    for (int e = 0; e < 25; ++e) {
      /* drop trailing exact zeros so len reports the true storage */
      int64_t L = P.len[e];
      if (L > cap) { rc = TIKH_ORACLE_EINVAL; break; }
      len[e] = L;
      cx* dst = (cx*)B + (size_t)e * (size_t)cap;
      for (int64_t t = 0; t < cap; ++t) dst[t] = (t < L) ? P.c[e][t] : 0.0;
    }
  }
  if (n_def) *n_def = nd;
  pm_free(&P);
  free(active);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Degree bounds (R10) and column scaling (R9).                                               */
/* ------------------------------------------------------------------------------------------ */

static void degree_bounds(int w, const int* din, const int* dout, int64_t* bound /* w * w */) {
  int have_active = 0, amax = 0;
  for (int j = 0; j < w; ++j)
    if (dout[j] > din[j]) {
      if (!have_active || dout[j] > amax) amax = dout[j];
      have_active = 1;
    }
  for (int i = 0; i < w; ++i)
    for (int j = 0; j < w; ++j) {
      int64_t b;
      if (dout[j] > din[j]) {
        b = (int64_t)dout[j] - din[i];
      } else {
        int64_t acc = have_active ? (int64_t)amax - din[i] : -1;
        if (i == j && acc < 0) acc = 0;
        int64_t tau_b = (int64_t)dout[j] - din[i];
        b = acc < tau_b ? acc : tau_b;
      }
      bound[w * i + j] = b;
    }
}

static int trim_to_bounds(pmat* B, const int64_t* bound) {
  for (int e = 0; e < B->w * B->w; ++e) {
    int64_t want = bound[e] < 0 ? 0 : bound[e] + 1;
    if (B->len[e] > want) {
      B->len[e] = want;
      if (want == 0) { free(B->c[e]); B->c[e] = NULL; }
    }
  }
  return 0;
}

static void scale_columns(pmat* B) {
  const int w = B->w;
  for (int j = 0; j < w; ++j) {
    double mx = 0.0;
    for (int i = 0; i < w; ++i) {
      int e = w * i + j;
      for (int64_t t = 0; t < B->len[e]; ++t) {
        double a = fabs(creal(B->c[e][t])), b = fabs(cimag(B->c[e][t]));
        if (a > mx) mx = a;
        if (b > mx) mx = b;
      }
    }
    if (mx == 0.0) continue;
    int ex;
    frexp(mx, &ex); /* mx = f 2^ex, f in [0.5, 1) */
    for (int i = 0; i < w; ++i) {
      int e = w * i + j;
      for (int64_t t = 0; t < B->len[e]; ++t)
        B->c[e][t] = ldexp(creal(B->c[e][t]), -ex) + ldexp(cimag(B->c[e][t]), -ex) * I;
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* The recursion (Algorithm 1 with paired interleaving, Sec. 6.1).                             */
/* A node is (a, s, L): its nodes are omega^{a + c + s j}, c in {0,1}, j < L; s L = N.         */
/* Its conditions, in list order, are position 2 ns j + ns c + f (f < ns: the condition set).  */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int64_t N, M;
  double eps;
  int mode;
  int w, ns;  /* basis size and condition sets per node */
  cx* R; /* residual rows [N][ns][w] */
  int64_t* deferred; /* deferred condition ids ns e + f */
  int64_t n_def, n_drop;
} rstate;

static int leaf_node(rstate* st, int64_t a, int64_t s, int64_t L, int* delta, pmat* out) {
  const int w = st->w, ns = st->ns;
  int K = (int)(2 * ns * L);
  cx* sig = (cx*)malloc(sizeof(cx) * (size_t)K);
  cx* r = (cx*)malloc(sizeof(cx) * (size_t)w * (size_t)K);
  char* act = (char*)malloc((size_t)K);
  int* dq = (int*)malloc(sizeof(int) * (size_t)K);
  int rc = TIKH_ORACLE_ENOMEM, nd = 0;
  if (!sig || !r || !act || !dq) goto done;
  for (int64_t j = 0; j < L; ++j)
    for (int c = 0; c < 2; ++c)
      for (int f = 0; f < ns; ++f) {
        int q = (int)(2 * ns * j + ns * c + f);
        int64_t e = a + c + s * j;
        sig[q] = node(e, st->N);
        memcpy(r + (size_t)w * q, st->R + ((size_t)ns * e + f) * w, sizeof(cx) * (size_t)w);
        act[q] = 1;
      }
  int din[WMAX];
  memcpy(din, delta, sizeof(int) * (size_t)w);
  if ((rc = pm_identity(out, w))) goto done;
  rc = serial_construct(K, sig, r, act, delta, st->eps, out, NULL, NULL, dq, &nd, &st->n_drop);
  if (rc) goto done;
  for (int i = 0; i < nd; ++i) {
    int q = dq[i];
    int64_t j = q / (2 * ns), c = (q / ns) % 2, f = q % ns;
    st->deferred[st->n_def++] = ns * (a + c + s * j) + f;
  }
  int64_t bound[WMAX * WMAX];
  degree_bounds(w, din, delta, bound);
  trim_to_bounds(out, bound);
  scale_columns(out);
done:
  free(sig); free(r); free(act); free(dq);
  return rc;
}

static int64_t smooth_at_least(int64_t v) {
  if (v < 1) v = 1;
  while (!is_5smooth(v)) ++v;
  return v;
}

/* step 2 of Algorithm 1: phi <- phi B_L(sigma) for every condition of the right child (aR, 2s, L/2) */
static int update_right(rstate* st, const pmat* BL, int64_t aR, int64_t sR, int64_t Lr) {
  const int w = st->w, ns = st->ns;
  int64_t N = st->N;
  int use_fft = st->mode == TIKH_ORACLE_FFT || (st->mode == TIKH_ORACLE_AUTO && Lr > 64);
  cx* val = (cx*)malloc(sizeof(cx) * (size_t)(w * w) * 2 * (size_t)Lr); /* [entry][c][j] */
  if (!val) return TIKH_ORACLE_ENOMEM;
  for (int e = 0; e < w * w; ++e)
    for (int c = 0; c < 2; ++c) {
      cx* v = val + ((size_t)e * 2 + c) * (size_t)Lr;
      int64_t beta = aR + c;
      if (!use_fft) {
        for (int64_t j = 0; j < Lr; ++j) v[j] = horner(BL->c[e], BL->len[e], node(beta + sR * j, N));
      } else {
        /* P(omega^{beta + sR j}) = sum_u g_u exp(2 pi i u j / Lr), g_u = sum_{t = u mod Lr} P_t omega^{beta t} */
        for (int64_t u = 0; u < Lr; ++u) v[u] = 0;
        for (int64_t t = 0; t < BL->len[e]; ++t) v[t % Lr] += BL->c[e][t] * node(beta * t, N);
        int rc = dft(v, Lr, +1);
        if (rc) { free(val); return rc; }
      }
    }
  for (int64_t j = 0; j < Lr; ++j)
    for (int c = 0; c < 2; ++c) {
      int64_t e = aR + c + sR * j;
      for (int f = 0; f < ns; ++f) {
        cx* rq = st->R + ((size_t)ns * e + f) * w;
        cx nr[WMAX];
        for (int col = 0; col < w; ++col) {
          cx acc = 0;
          for (int i = 0; i < w; ++i) acc += rq[i] * val[((size_t)(w * i + col) * 2 + c) * (size_t)Lr + j];
          nr[col] = acc;
        }
        memcpy(rq, nr, sizeof(cx) * (size_t)w);
      }
    }
  free(val);
  return 0;
}

/* step 4 of Algorithm 1: B = B_L B_R, trimmed to the node's degree bounds */
static int multiply(const rstate* st, const pmat* BL, const pmat* BR, const int64_t* bound, pmat* out) {
  const int w = BL->w;
  memset(out, 0, sizeof(*out));
  out->w = w;
  int64_t D = -1;
  for (int e = 0; e < w * w; ++e)
    if (bound[e] > D) D = bound[e];
  int64_t maxlen = 0;
  for (int e = 0; e < w * w; ++e) {
    if (BL->len[e] > maxlen) maxlen = BL->len[e];
    if (BR->len[e] > maxlen) maxlen = BR->len[e];
  }
  int use_fft = st->mode == TIKH_ORACLE_FFT || (st->mode == TIKH_ORACLE_AUTO && maxlen > 64);
  if (!use_fft) {
    for (int i = 0; i < w; ++i)
      for (int j = 0; j < w; ++j) {
        int eo = w * i + j;
        int64_t want = bound[eo] < 0 ? 0 : bound[eo] + 1;
        if (want == 0) continue;
        if (pm_reserve(out, eo, want)) return TIKH_ORACLE_ENOMEM;
        for (int t = 0; t < w; ++t) {
          const cx* x = BL->c[w * i + t];
          const cx* y = BR->c[w * t + j];
          int64_t lx = BL->len[w * i + t], ly = BR->len[w * t + j];
          for (int64_t u = 0; u < lx; ++u)
            for (int64_t v = 0; v < ly; ++v)
              if (u + v < want) out->c[eo][u + v] += x[u] * y[v];
        }
      }
    return 0;
  }
  /* FFT products of length P > D: a linear convolution of polynomials whose product has degree
   * <= D equals the cyclic one */
  int64_t P = smooth_at_least(D + 1);
  cx* fl = (cx*)calloc((size_t)(w * w) * (size_t)P, sizeof(cx));
  cx* fr = (cx*)calloc((size_t)(w * w) * (size_t)P, sizeof(cx));
  cx* acc = (cx*)malloc(sizeof(cx) * (size_t)P);
  int rc = TIKH_ORACLE_ENOMEM;
  if (!fl || !fr || !acc) goto done;
  for (int e = 0; e < w * w; ++e) {
    /* entries longer than P would wrap; their high coefficients multiply into terms above D
     * only if the bound is violated, which trim_to_bounds would have removed anyway */
    int64_t lx = BL->len[e] < P ? BL->len[e] : P, ly = BR->len[e] < P ? BR->len[e] : P;
    for (int64_t t = 0; t < lx; ++t) fl[(size_t)e * P + t] = BL->c[e][t];
    for (int64_t t = 0; t < ly; ++t) fr[(size_t)e * P + t] = BR->c[e][t];
    if (lx && (rc = dft(fl + (size_t)e * P, P, +1))) goto done;
    if (ly && (rc = dft(fr + (size_t)e * P, P, +1))) goto done;
  }
  for (int i = 0; i < w; ++i)
    for (int j = 0; j < w; ++j) {
      int eo = w * i + j;
      int64_t want = bound[eo] < 0 ? 0 : bound[eo] + 1;
      if (want == 0) continue;
      for (int64_t u = 0; u < P; ++u) {
        cx s = 0;
        for (int t = 0; t < w; ++t) s += fl[(size_t)(w * i + t) * P + u] * fr[(size_t)(w * t + j) * P + u];
        acc[u] = s;
      }
      if ((rc = dft(acc, P, -1))) goto done;
      if (pm_reserve(out, eo, want)) { rc = TIKH_ORACLE_ENOMEM; goto done; }
      for (int64_t u = 0; u < want; ++u) out->c[eo][u] = acc[u] / (double)P;
    }
  rc = 0;
done:
  free(fl); free(fr); free(acc);
  return rc;
}

static int rec_tanint(rstate* st, int64_t a, int64_t s, int64_t L, int* delta, pmat* out) {
  if (2 * L == st->M) return leaf_node(st, a, s, L, delta, out);
  const int w = st->w;
  int din[WMAX];
  memcpy(din, delta, sizeof(int) * (size_t)w);
  pmat BL, BR;
  memset(&BR, 0, sizeof(BR));
  int rc = rec_tanint(st, a, 2 * s, L / 2, delta, &BL); /* step 1: {t mod 4 in {0,1}} */
  if (rc) return rc;
  rc = update_right(st, &BL, a + s, 2 * s, L / 2); /* step 2 */
  if (!rc) rc = rec_tanint(st, a + s, 2 * s, L / 2, delta, &BR); /* step 3: {t mod 4 in {2,3}} */
  if (!rc) {
    int64_t bound[WMAX * WMAX];
    degree_bounds(w, din, delta, bound);
    rc = multiply(st, &BL, &BR, bound, out); /* step 4 */
    if (!rc) scale_columns(out);
  }
  pm_free(&BL);
  pm_free(&BR);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Drivers.                                                                                   */
/* ------------------------------------------------------------------------------------------ */

int tikh_oracle_conditions(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                           double lam, const tikh_oracle_opts* opts, double* F, double* G, int* tau) {
  int64_t N, M, k;
  int p;
  int rc = tikh_oracle_plan(m, n, opts, &N, &M, &k, &p);
  if (rc) return rc;
  rc = build_conditions(m, n, N, k, (const cx*)col, (const cx*)row, (const cx*)y, lam, opts->fill, opts->is_complex,
                        (cx*)F, (cx*)G);
  if (rc) return rc;
  tau[0] = (int)(n - 1); tau[1] = (int)(m - 1); tau[2] = (int)(m + k - 2); tau[3] = (int)(n + k - 2); tau[4] = 0;
  return 0;
}

int tikh_oracle_solve_normal(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                             double lam, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats,
                             double* Bout, int64_t cap, int64_t* lenout) {
  return tikh_oracle_solve_normal_ex(m, n, col, row, y, lam, opts, x, stats, Bout, cap, lenout, NULL, 0);
}

/* x-column of the first block row of the Toeplitz-Gramian system (Sec. 3.4, Eq. (gramblk)): the n x n
 * Hermitian Toeplitz G (G[i][j] = g_{i-j}, g_{-d} = conj(g_d)) below N-n extension rows.  Its circulant
 * generator is c11[(N-n+d) mod N] = g_d for |d| <= n-1; the other N-2n+1 entries are the arbitrary
 * extension entries, filled as in R5 (peak of g times SplitMix64 uniforms, counters offset by 2^40 so they
 * differ from L's).  Returns DFT(c11) (positive exponent) in out (N entries). */
static int gram_column(int64_t n, int64_t N, const cx* g, int fill, int is_complex, cx* out) {
  cx* gt = (cx*)malloc(sizeof(cx) * (size_t)N); /* gt[d mod N] = g_d */
  if (!gt) return TIKH_ORACLE_ENOMEM;
  for (int64_t d = 0; d < N; ++d) gt[d] = 0;
  for (int64_t d = 0; d < n; ++d) gt[d] = g[d];
  for (int64_t d = 1; d < n; ++d) gt[N - d] = conj(g[d]);
  const int64_t nfill = N - 2 * n + 1; /* indices n .. N-n */
  double peak = 0.0;
  for (int64_t d = 0; d < n; ++d) {
    if (fabs(creal(g[d])) > peak) peak = fabs(creal(g[d]));
    if (fabs(cimag(g[d])) > peak) peak = fabs(cimag(g[d]));
  }
  for (int64_t i = 1; i <= nfill; ++i) {
    cx v;
    if (fill == 1) {
      v = g[n - 1] + (conj(g[n - 1]) - g[n - 1]) * ((double)i / (double)(nfill + 1));
    } else {
      double re = peak * splitmix_uniform((uint64_t)(2 * i) + (1ULL << 40));
      double im = is_complex ? peak * splitmix_uniform((uint64_t)(2 * i + 1) + (1ULL << 40)) : 0.0;
      v = re + im * I;
    }
    gt[n - 1 + i] = v;
  }
  for (int64_t j = 0; j < N; ++j) out[j] = gt[((j - (N - n)) % N + N) % N];
  free(gt);
  return dft(out, N, +1);
}

/* The superfast solve from given conditions: cond[N][ns][w] (row f of node e: the condition of set f at
 * omega^e), tau[w] (Eq. (taudef); the starting basis I has tau-degrees -tau), the plan (N, M).  Algorithm 1
 * over all N nodes, the difficult points at the end (Sec. 5), extraction x(z) = B*_{1,j}(z) / B*_{w,j}
 * for the column j of tau-degree 0 (Sec. 4.3 end, Sec. 5): nx coefficients of x. */
static int solve_conditions(int64_t N, int64_t M, int w, int ns, const cx* cond, const int* tau, int64_t nx,
                            const tikh_oracle_opts* opts, cx* x, int* delta_out, int64_t* n_def, int64_t* n_drop,
                            double* Bout, int64_t cap, int64_t* lenout, int64_t* deferred_out,
                            int64_t deferred_cap) {
  rstate st;
  memset(&st, 0, sizeof(st));
  st.N = N; st.M = M; st.eps = opts->eps_diff; st.mode = opts->mode; st.w = w; st.ns = ns;
  const size_t rows = (size_t)ns * (size_t)N;
  st.R = (cx*)malloc(sizeof(cx) * rows * (size_t)w);
  st.deferred = (int64_t*)malloc(sizeof(int64_t) * rows);
  pmat B;
  memset(&B, 0, sizeof(B));
  int rc = TIKH_ORACLE_ENOMEM;
  if (!st.R || !st.deferred) goto done;
  memcpy(st.R, cond, sizeof(cx) * rows * (size_t)w);
  int delta[WMAX];
  for (int i = 0; i < w; ++i) delta[i] = -tau[i];
  /* root node: all N nodes = omega^{0 + c + 2 j}, j < N/2 */
  if ((rc = rec_tanint(&st, 0, 2, N / 2, delta, &B))) goto done;
  if (deferred_out)
    for (int64_t q = 0; q < st.n_def && q < deferred_cap; ++q) deferred_out[q] = st.deferred[q];
  if (st.n_def > 0) {
    /* difficult points (Sec. 5): residual against the final basis, then serial processing */
    int K = (int)st.n_def;
    cx* sig = (cx*)malloc(sizeof(cx) * (size_t)K);
    cx* r = (cx*)malloc(sizeof(cx) * (size_t)w * (size_t)K);
    char* act = (char*)malloc((size_t)K);
    if (!sig || !r || !act) { free(sig); free(r); free(act); rc = TIKH_ORACLE_ENOMEM; goto done; }
    for (int q = 0; q < K; ++q) {
      int64_t id = st.deferred[q], e = id / ns;
      const cx* ph = cond + ((size_t)ns * e + (size_t)(id % ns)) * w;
      sig[q] = node(e, N);
      for (int j = 0; j < w; ++j) {
        cx acc = 0;
        for (int i = 0; i < w; ++i) acc += ph[i] * horner(B.c[w * i + j], B.len[w * i + j], sig[q]);
        r[w * q + j] = acc;
      }
      act[q] = 1;
    }
    rc = serial_construct(K, sig, r, act, delta, -1.0, &B, NULL, NULL, NULL, NULL, &st.n_drop);
    free(sig); free(r); free(act);
    if (rc) goto done;
  }
  /* Sec. 4.3 end: one column has tau-degree 0, the other w - 1 have 1 */
  int jstar = -1, nzero = 0, none = 0;
  for (int j = 0; j < w; ++j) {
    if (delta[j] == 0) { jstar = j; ++nzero; }
    else if (delta[j] == 1) ++none;
  }
  memcpy(delta_out, delta, sizeof(int) * (size_t)w);
  *n_def = st.n_def;
  *n_drop = st.n_drop;
  if (nzero != 1 || none != w - 1 || B.len[w * (w - 1) + jstar] < 1) { rc = TIKH_ORACLE_ENUMERIC; goto done; }
  {
    cx cw = B.c[w * (w - 1) + jstar][0];
    const cx* b1 = B.c[jstar];
    int64_t l1 = B.len[jstar];
    for (int64_t i = 0; i < nx; ++i) x[i] = (i < l1 ? b1[i] : 0.0) / cw;
  }
  if (Bout && lenout) {
    for (int e = 0; e < w * w; ++e) {
      int64_t L = B.len[e] < cap ? B.len[e] : cap;
      lenout[e] = B.len[e];
      cx* dst = (cx*)Bout + (size_t)e * (size_t)cap;
      for (int64_t t = 0; t < cap; ++t) dst[t] = (t < L) ? B.c[e][t] : 0.0;
    }
  }
  rc = 0;
done:
  pm_free(&B);
  free(st.R); free(st.deferred);
  return rc;
}

/* The l2 system (Eq. (ex6)) for (T^H T + lam I) x = y, or with gram != NULL the Toeplitz-Gramian system
 * (Eq. (ex7)) for (G + L^H L) x = y with L = [col, row] (m x n) in the role of T and G (first column gram)
 * in place of lam I: conditions F, G (two sets), tau = [n-1, m-1, m+k-2, n+k-2, 0], then the solve. */
static int solve_core(int64_t m, int64_t n, const double* col, const double* row, const double* y, double lam,
                      const double* gram, int64_t N, int64_t M, int64_t k, int p, const tikh_oracle_opts* opts,
                      double* x, tikh_oracle_stats* stats, double* Bout, int64_t cap, int64_t* lenout,
                      int64_t* deferred_out, int64_t deferred_cap) {
  cx* F = (cx*)malloc(sizeof(cx) * 5 * (size_t)N);
  cx* G = (cx*)malloc(sizeof(cx) * 5 * (size_t)N);
  cx* cond = (cx*)malloc(sizeof(cx) * 10 * (size_t)N);
  int rc = TIKH_ORACLE_ENOMEM;
  if (!F || !G || !cond) goto done;
  if ((rc = build_conditions(m, n, N, k, (const cx*)col, (const cx*)row, (const cx*)y, lam, opts->fill,
                             opts->is_complex, F, G)))
    goto done;
  if (gram) { /* Toeplitz-Gramian: F's x component is the DFT of G's generator instead of lam w^{e(m+k-1)} */
    cx* c11 = (cx*)malloc(sizeof(cx) * (size_t)N);
    if (!c11) { rc = TIKH_ORACLE_ENOMEM; goto done; }
    rc = gram_column(n, N, (const cx*)gram, opts->fill, opts->is_complex, c11);
    for (int64_t e = 0; e < N && !rc; ++e) F[5 * e] = c11[e];
    free(c11);
    if (rc) goto done;
  }
  for (int64_t e = 0; e < N; ++e) {
    memcpy(cond + 10 * e, F + 5 * e, sizeof(cx) * 5);
    memcpy(cond + 10 * e + 5, G + 5 * e, sizeof(cx) * 5);
  }
  {
    /* Eq. (taudef) with reading R3 */
    int tau[5] = {(int)(n - 1), (int)(m - 1), (int)(m + k - 2), (int)(n + k - 2), 0};
    int delta[5];
    int64_t nd = 0, ndrop = 0;
    rc = solve_conditions(N, M, 5, 2, cond, tau, n, opts, (cx*)x, delta, &nd, &ndrop, Bout, cap, lenout, deferred_out,
                          deferred_cap);
    if (stats) {
      stats->N = N; stats->M = M; stats->k = k; stats->p = p;
      stats->n_difficult = nd; stats->n_dropped = ndrop;
      memcpy(stats->delta, delta, sizeof(delta));
      stats->jstar = -1;
      for (int j = 0; j < 5; ++j)
        if (delta[j] == 0) stats->jstar = j;
      stats->dual = 0;
    }
  }
done:
  free(F); free(G); free(cond);
  return rc;
}

int tikh_oracle_solve_normal_ex(int64_t m, int64_t n, const double* col, const double* row, const double* y,
                                double lam, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats,
                                double* Bout, int64_t cap, int64_t* lenout, int64_t* deferred_out,
                                int64_t deferred_cap) {
  int64_t N, M, k;
  int p;
  int rc = tikh_oracle_plan(m, n, opts, &N, &M, &k, &p);
  if (rc) return rc;
  return solve_core(m, n, col, row, y, lam, NULL, N, M, k, p, opts, x, stats, Bout, cap, lenout, deferred_out,
                    deferred_cap);
}

/* Sec. 3.4: q = max(n, pl); Algorithm 2 sizes N >= q + n - 1 (so the N-n extension rows of the first
 * block row hold G's generator, N - 2n + 1 >= 0), and L's extension is k = N - (pl + n - 1). */
int tikh_oracle_solve_gramian(int64_t n, int64_t pl, const double* g, const double* lcol, const double* lrow,
                              const double* y, const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats) {
  if (n < 1 || pl < 1 || !opts) return TIKH_ORACLE_EINVAL;
  const int64_t q = n > pl ? n : pl;
  int64_t N, M, k0;
  int p;
  int rc = tikh_oracle_plan(q, n, opts, &N, &M, &k0, &p);
  if (rc) return rc;
  const int64_t k = N - (pl + n - 1);
  return solve_core(pl, n, lcol, lrow, y, 0.0, g, N, M, k, p, opts, x, stats, NULL, 0, NULL, NULL, 0);
}

/* ------------------------------------------------------------------------------------------ */
/* The general problem (Sec. 3.2, Eq. (ex1)-(ex3)): (T^H T + L^H L) x = y with T (m x n) and     */
/* L (p x n) generic Toeplitz.  Reading R22: all three block rows are extended to the same N     */
/* points (the nodes are shared), N >= max(m, p) + n - 1, so block row 1 has N - n extension rows, */
/* block row 2 N - m and block row 3 N - p; gamma_1, gamma_2, gamma_3 have those lengths.         */
/* ------------------------------------------------------------------------------------------ */

/* Conditions F, G, H per node (Eq. (interp)), rows cond[N][3][7] over the unknowns
 *   [x (n), sigma_1 (m), sigma_2 (p), gamma_1 (N-n), gamma_2 (N-m), gamma_3 (N-p), 1]:
 *   block row 1: T^H sigma_1 + L^H sigma_2 - y = 0 below N-n rows defining gamma_1
 *   block row 2: -T x + sigma_1 = 0 below N-m rows defining gamma_2
 *   block row 3: -L x + sigma_2 = 0 below N-p rows defining gamma_3
 * each partial circulant turned into the DFT of its generator (Eq. (circdiag)). */
static int build_conditions_general(int64_t m, int64_t n, int64_t p, int64_t N, const cx* col, const cx* row,
                                    const cx* lcol, const cx* lrow, const cx* y, int fill, int is_complex,
                                    cx* cond) {
  const int64_t kT = N - (m + n - 1), kL = N - (p + n - 1);
  cx* aT = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* aL = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cT = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cH = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cL = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cLH = (cx*)malloc(sizeof(cx) * (size_t)N);
  cx* cy = (cx*)malloc(sizeof(cx) * (size_t)N);
  int rc = TIKH_ORACLE_ENOMEM;
  if (!aT || !aL || !cT || !cH || !cL || !cLH || !cy) goto done;
  periodic_generator(m, n, N, kT, col, row, fill, is_complex, 0, aT);
  periodic_generator(p, n, N, kL, lcol, lrow, fill, is_complex, 1ULL << 41, aL);
  for (int64_t j = 0; j < N; ++j) {
    cT[j] = aT[((j - (N - m)) % N + N) % N];        /* C(T): rows N-m .. N-1 hold T       (R2) */
    cL[j] = aL[((j - (N - p)) % N + N) % N];        /* C(L): rows N-p .. N-1 hold L            */
    cH[j] = conj(aT[((N - n - j) % N + N) % N]);    /* C(T^H): rows N-n .. N-1 hold T^H        */
    cLH[j] = conj(aL[((N - n - j) % N + N) % N]);   /* C(L^H): rows N-n .. N-1 hold L^H        */
    cy[j] = 0;
  }
  for (int64_t i = 0; i < n; ++i) cy[N - n + i] = -y[i];
  if ((rc = dft(cT, N, +1)) || (rc = dft(cL, N, +1)) || (rc = dft(cH, N, +1)) || (rc = dft(cLH, N, +1)) ||
      (rc = dft(cy, N, +1)))
    goto done;
  for (int64_t e = 0; e < N; ++e) {
    cx* f = cond + 21 * e;
    cx* g = f + 7;
    cx* h = f + 14;
    for (int i = 0; i < 21; ++i) f[i] = 0.0;
    f[1] = cH[e];               /* C_12 */
    f[2] = cLH[e];              /* C_13 */
    f[3] = 1.0;                 /* C_14 = [I_{N-n}; 0]: generator e_0 */
    f[6] = cy[e];               /* C_17 */
    g[0] = -cT[e];              /* C_21 */
    g[1] = node(e * (N - m), N); /* C_22 = [0; I_m] below N-m rows: generator e_{N-m} */
    g[4] = 1.0;                 /* C_25 */
    h[0] = -cL[e];              /* C_31 */
    h[2] = node(e * (N - p), N); /* C_33 */
    h[5] = 1.0;                 /* C_36 */
  }
  rc = 0;
done:
  free(aT); free(aL); free(cT); free(cH); free(cL); free(cLH); free(cy);
  return rc;
}

/* Algorithm 2 with three condition sets per node over N >= max(m, p) + n - 1 */
int tikh_oracle_plan_general(int64_t m, int64_t n, int64_t p, const tikh_oracle_opts* opts, int64_t* N, int64_t* M,
                             int* pp) {
  if (m < 1 || n < 1 || p < 1 || !opts) return TIKH_ORACLE_EINVAL;
  const int64_t q = m > p ? m : p;
  return plan_sets(q + n - 1, 3, opts, N, M, pp);
}

int tikh_oracle_conditions_general(int64_t m, int64_t n, int64_t p, const double* col, const double* row,
                                   const double* lcol, const double* lrow, const double* y,
                                   const tikh_oracle_opts* opts, double* cond, int* tau) {
  int64_t N, M;
  int pp;
  int rc = tikh_oracle_plan_general(m, n, p, opts, &N, &M, &pp);
  if (rc) return rc;
  rc = build_conditions_general(m, n, p, N, (const cx*)col, (const cx*)row, (const cx*)lcol, (const cx*)lrow,
                                (const cx*)y, opts->fill, opts->is_complex, (cx*)cond);
  if (rc) return rc;
  /* Eq. (taudef) for unequal sizes: tau_i + 1 = the length of unknown i */
  tau[0] = (int)(n - 1); tau[1] = (int)(m - 1); tau[2] = (int)(p - 1);
  tau[3] = (int)(N - n - 1); tau[4] = (int)(N - m - 1); tau[5] = (int)(N - p - 1); tau[6] = 0;
  return 0;
}

int tikh_oracle_solve_general(int64_t m, int64_t n, int64_t p, const double* col, const double* row,
                              const double* lcol, const double* lrow, const double* y, const tikh_oracle_opts* opts,
                              double* x, tikh_oracle_stats* stats) {
  int64_t N, M;
  int pp;
  int rc = tikh_oracle_plan_general(m, n, p, opts, &N, &M, &pp);
  if (rc) return rc;
  cx* cond = (cx*)malloc(sizeof(cx) * 21 * (size_t)N);
  if (!cond) return TIKH_ORACLE_ENOMEM;
  int tau[7];
  rc = tikh_oracle_conditions_general(m, n, p, col, row, lcol, lrow, y, opts, (double*)cond, tau);
  if (!rc) {
    int delta[7];
    int64_t nd = 0, ndrop = 0;
    rc = solve_conditions(N, M, 7, 3, cond, tau, n, opts, (cx*)x, delta, &nd, &ndrop, NULL, 0, NULL, NULL, 0);
    if (stats) {
      stats->N = N; stats->M = M; stats->k = N - (m + n - 1); stats->p = pp;
      stats->n_difficult = nd; stats->n_dropped = ndrop;
      memcpy(stats->delta, delta, sizeof(delta));
      stats->jstar = -1;
      for (int j = 0; j < 7; ++j)
        if (delta[j] == 0) stats->jstar = j;
      stats->dual = 0;
    }
  }
  free(cond);
  return rc;
}

/* y = T^H v and u = T x through the circulant embedding of length >= m+n-1 (a plain DFT identity) */
static int toeplitz_apply(int64_t m, int64_t n, const cx* col, const cx* row, const cx* in, cx* out, int herm) {
  int64_t L = smooth_at_least(m + n - 1);
  cx* g = (cx*)calloc((size_t)L, sizeof(cx));
  cx* v = (cx*)calloc((size_t)L, sizeof(cx));
  int rc = TIKH_ORACLE_ENOMEM;
  if (!g || !v) goto done;
  if (!herm) {
    /* (T x)_i = sum_j a_{i-j} x_j: cyclic convolution of g[d mod L] = a_d with x */
    for (int64_t d = 0; d < m; ++d) g[d] = col[d];
    for (int64_t d = 1; d < n; ++d) g[L - d] = row[d];
    for (int64_t j = 0; j < n; ++j) v[j] = in[j];
  } else {
    /* (T^H v)_i = sum_j conj(a_{j-i}) v_j: g[d mod L] = conj(a_{-d}) for d in [-(m-1), n-1] */
    for (int64_t d = 0; d < n; ++d) g[d] = conj(d == 0 ? col[0] : row[d]);
    for (int64_t d = 1; d < m; ++d) g[L - d] = conj(col[d]);
    for (int64_t j = 0; j < m; ++j) v[j] = in[j];
  }
  if ((rc = dft(g, L, +1)) || (rc = dft(v, L, +1))) goto done;
  for (int64_t t = 0; t < L; ++t) v[t] *= g[t];
  if ((rc = dft(v, L, -1))) goto done;
  for (int64_t i = 0; i < (herm ? n : m); ++i) out[i] = v[i] / (double)L;
  rc = 0;
done:
  free(g); free(v);
  return rc;
}

int tikh_oracle_apply_th(int64_t m, int64_t n, const double* col, const double* row, const double* v, double* y) {
  if (m < 1 || n < 1) return TIKH_ORACLE_EINVAL;
  return toeplitz_apply(m, n, (const cx*)col, (const cx*)row, (const cx*)v, (cx*)y, 1);
}

int tikh_oracle_apply_t(int64_t m, int64_t n, const double* col, const double* row, const double* x, double* u) {
  if (m < 1 || n < 1) return TIKH_ORACLE_EINVAL;
  return toeplitz_apply(m, n, (const cx*)col, (const cx*)row, (const cx*)x, (cx*)u, 0);
}

int tikh_oracle_solve(int64_t m, int64_t n, const double* col, const double* row, const double* b, double lam,
                      const tikh_oracle_opts* opts, double* x, tikh_oracle_stats* stats) {
  if (m < 1 || n < 1 || !(lam > 0.0) || !opts) return TIKH_ORACLE_EINVAL;
  int rc;
  if (m >= n) {
    cx* y = (cx*)malloc(sizeof(cx) * (size_t)n);
    if (!y) return TIKH_ORACLE_ENOMEM;
    rc = tikh_oracle_apply_th(m, n, col, row, b, (double*)y);
    if (!rc) rc = tikh_oracle_solve_normal(m, n, col, row, (const double*)y, lam, opts, x, stats, NULL, 0, NULL);
    free(y);
    return rc;
  }
  /* R11: T' = T^H is n x m with a'_d = conj(a_{-d}): col'[d] = conj(row[d]) (d >= 1),
   * col'[0] = conj(a_0), row'[d] = conj(col[d]) */
  cx* cp = (cx*)malloc(sizeof(cx) * (size_t)n);
  cx* rp = (cx*)malloc(sizeof(cx) * (size_t)m);
  cx* v = (cx*)malloc(sizeof(cx) * (size_t)m);
  rc = TIKH_ORACLE_ENOMEM;
  if (cp && rp && v) {
    const cx* c = (const cx*)col;
    const cx* r = (const cx*)row;
    cp[0] = conj(c[0]);
    for (int64_t d = 1; d < n; ++d) cp[d] = conj(r[d]);
    for (int64_t d = 0; d < m; ++d) rp[d] = conj(c[d]);
    rc = tikh_oracle_solve_normal(n, m, (const double*)cp, (const double*)rp, b, lam, opts, (double*)v, stats, NULL,
                                  0, NULL);
    if (!rc) rc = tikh_oracle_apply_th(m, n, col, row, (const double*)v, x);
    if (stats) stats->dual = 1;
  }
  free(cp); free(rp); free(v);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Iterative refinement (Sec. 7.2 notes that the direct solution "can be further improved with  */
/* iterative refinement"): on the core system A v = y, A = T_c^H T_c + lam I (T_c the tall core */
/* matrix, y its right-hand side), v <- v + A^{-1}(y - A v), each correction by the same        */
/* superfast solve with the residual as right-hand side.                                       */
/* ------------------------------------------------------------------------------------------ */

int tikh_oracle_solve_refined(int64_t m, int64_t n, const double* col, const double* row, const double* b,
                              double lam, const tikh_oracle_opts* opts, int steps, double* x, tikh_oracle_stats* stats,
                              double* rel_residual) {
  if (m < 1 || n < 1 || !(lam > 0.0) || !opts || steps < 0) return TIKH_ORACLE_EINVAL;
  int dual = m < n;
  int64_t cm = dual ? n : m, cn = dual ? m : n;
  cx* cc = (cx*)malloc(sizeof(cx) * (size_t)cm);
  cx* cr = (cx*)malloc(sizeof(cx) * (size_t)cn);
  cx* y = (cx*)malloc(sizeof(cx) * (size_t)cn);
  cx* v = (cx*)malloc(sizeof(cx) * (size_t)cn);
  cx* dv = (cx*)malloc(sizeof(cx) * (size_t)cn);
  cx* r = (cx*)malloc(sizeof(cx) * (size_t)cn);
  cx* u = (cx*)malloc(sizeof(cx) * (size_t)cm);
  int rc = TIKH_ORACLE_ENOMEM;
  if (!cc || !cr || !y || !v || !dv || !r || !u) goto done;
  if (!dual) {
    memcpy(cc, col, sizeof(cx) * (size_t)m);
    memcpy(cr, row, sizeof(cx) * (size_t)n);
    if ((rc = tikh_oracle_apply_th(m, n, col, row, b, (double*)y))) goto done;
  } else { /* core matrix T^H: a'_d = conj(a_{-d}) */
    const cx* c = (const cx*)col;
    const cx* rw = (const cx*)row;
    cc[0] = conj(c[0]);
    for (int64_t d = 1; d < cm; ++d) cc[d] = conj(rw[d]);
    for (int64_t d = 0; d < cn; ++d) cr[d] = conj(c[d]);
    memcpy(y, b, sizeof(cx) * (size_t)cn);
  }
  if ((rc = tikh_oracle_solve_normal(cm, cn, (double*)cc, (double*)cr, (double*)y, lam, opts, (double*)v, stats, NULL,
                                     0, NULL)))
    goto done;
  double ny = 0.0, nr = 0.0;
  for (int64_t i = 0; i < cn; ++i) ny += creal(y[i]) * creal(y[i]) + cimag(y[i]) * cimag(y[i]);
  for (int it = 0; it <= steps; ++it) {
    /* r = y - (T_c^H (T_c v) + lam v) */
    if ((rc = tikh_oracle_apply_t(cm, cn, (double*)cc, (double*)cr, (double*)v, (double*)u))) goto done;
    if ((rc = tikh_oracle_apply_th(cm, cn, (double*)cc, (double*)cr, (double*)u, (double*)r))) goto done;
    nr = 0.0;
    for (int64_t i = 0; i < cn; ++i) {
      r[i] = y[i] - (r[i] + lam * v[i]);
      nr += creal(r[i]) * creal(r[i]) + cimag(r[i]) * cimag(r[i]);
    }
    if (it == steps) break;
    if ((rc = tikh_oracle_solve_normal(cm, cn, (double*)cc, (double*)cr, (double*)r, lam, opts, (double*)dv, NULL,
                                       NULL, 0, NULL)))
      goto done;
    for (int64_t i = 0; i < cn; ++i) v[i] += dv[i];
  }
  if (rel_residual) *rel_residual = ny > 0.0 ? sqrt(nr / ny) : sqrt(nr);
  if (!dual) memcpy(x, v, sizeof(cx) * (size_t)n);
  else rc = tikh_oracle_apply_th(m, n, col, row, (double*)v, x);
  if (stats) stats->dual = dual;
done:
  free(cc); free(cr); free(y); free(v); free(dv); free(r); free(u);
  return rc;
}
