// internal.h -- plan structure and kernel launchers shared by the translation units of libtikh.
#pragma once
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/tikh.h"
#include "common.cuh"
#include "fft.cuh"

namespace tikh {

constexpr int MAX_DEPTH = 40;

// one basis matrix B(z): 25 polynomials (entry (i,j) at c + (5i+j)*cap), device-side lengths and the
// per-column max |Re|,|Im| (bit pattern) that fixes the lazy power-of-two column scaling
struct BasisBuf {
  cd* c = nullptr;
  int* len = nullptr;                   // 25
  unsigned long long* colmax = nullptr;  // 5
  int64_t cap = 0;
};

// DFS schedule of Algorithm 1: a node (a, s, L) at `depth` has nodes omega^{a + c + s j}, c in {0,1},
// j < L (s L = N) and 4L conditions.
enum StepKind { STEP_LEAF = 0, STEP_EVAL = 1, STEP_PROD = 2 };
struct Step {
  int kind;
  int depth;
  int side;  // 0: left child (writes buf[depth][0]), 1: right child
  int64_t a, s, L;
  int fft;          // FFT plan index: eval length L/2 (STEP_EVAL) or product length P (STEP_PROD)
  int64_t P;        // product transform length (STEP_PROD)
  uint64_t save_mask;  // STEP_LEAF: depths whose delta_in is this leaf's delta_in
};

struct Plan {
  // problem
  int64_t m = 0, n = 0;
  int dtype = 0;
  tikh_opts opts{};
  cudaStream_t stream = nullptr;
  int dual = 0;
  int64_t cm = 0, cn = 0;  // core (tall) problem: cm >= cn
  int64_t N = 0, M = 0, k = 0;
  int p = 0;
  int slack_mult = 1;  // degree-prediction slack multiplier (raised after TIKH_EDEGREE)

  std::vector<Step> sched;
  std::map<int64_t, int> fft_of_len;
  std::vector<FftPlan> ffts;
  std::map<int64_t, cd*> twiddle_of_len;
  int64_t Pmax = 0, Lrmax = 0;

  // device memory
  std::vector<void*> allocs;
  int64_t bytes = 0;
  cd* wN = nullptr;     // omega^e, e < N
  cd* specT = nullptr;  // DFT of the circulant generator of the core T
  cd* work = nullptr;   // N
  cd* work2 = nullptr;  // N
  cd* ftmpN = nullptr;  // N (four-step temp for length-N transforms)
  cd* R = nullptr;      // residual rows [N][2][5]
  cd* Phi = nullptr;    // original condition rows [N][2][5]
  int* delta = nullptr;   // 5
  int* dstack = nullptr;  // MAX_DEPTH * 5
  int* status = nullptr;  // 1
  int* ndiff = nullptr;   // 1
  int64_t* diff = nullptr;  // max_difficult condition ids 2e + f
  cd* diffr = nullptr;      // max_difficult * 5 residuals
  BasisBuf buf[MAX_DEPTH][2];
  cd* evalv = nullptr;  // 50 * Lrmax
  cd* etmp = nullptr;   // 50 * Lrmax (four-step temp)
  cd* FA = nullptr;     // 25 * Pmax spectra of B_L
  cd* FB = nullptr;     // 25 * Pmax spectra of B_R
  cd* FC = nullptr;     // 25 * Pmax products
  cd* ptmp = nullptr;   // 50 * Pmax (four-step temp)
  unsigned long long* peak = nullptr;  // fill magnitude (bit pattern of a non-negative double)
  cd* ybuf = nullptr;    // core right-hand side (cn)
  cd* rbuf = nullptr;    // refinement residual (cn)
  cd* xcore = nullptr;   // core solution (cn)
  cd* dx = nullptr;      // refinement correction (cn)
  double* norms = nullptr;  // ||r||^2, ||y||^2 of the last residual
  cd* dscr = nullptr;    // difficult-point scratch: 5 * buf[0][0].cap + max_difficult
  void* d_in = nullptr;  // staging for tikh_solve_host: col | row | b | x
  int64_t launches = 0;

  tikh_stats last{};
};

// launchers (return the number of kernels enqueued, or a negative TIKH_E* code)
int launch_twiddle(cd* tab, int64_t L, cudaStream_t s);
int launch_spectrum(Plan& P, const void* col, const void* row);
int launch_rhs(Plan& P, const void* rhs, int rhs_is_y);
int launch_conditions(Plan& P, const cd* y, double lam);
int launch_extract(Plan& P, cd* out);
int launch_residual(Plan& P, const cd* y, const cd* x, cd* r, double lam);
int launch_axpy(Plan& P, cd* x, const cd* dx);
int launch_output(Plan& P, const cd* v, void* x);
int launch_leaf(Plan& P, const Step& st, int nlim_threads);
int launch_eval(Plan& P, const Step& st);
int launch_prod(Plan& P, const Step& st);
int launch_difficult(Plan& P);
int launch_leaf_arrays(int K, const cd* sigma, const cd* r, int* delta, double eps, cd* B, int* len,
                       unsigned long long* colmax, int* ndiff, int64_t* diff, int* status, int* order, int* pivot,
                       cudaStream_t s);
int launch_fft_test(int64_t L, cd* data, int sign, cudaStream_t s, int64_t* bytes_out);

}  // namespace tikh
