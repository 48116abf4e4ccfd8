// internal.h -- plan structure and kernel launchers shared by the translation units of libtikh.
//
// Every per-problem device array carries a leading problem index: a plan is built for up to
// `batch_max` problems of the same shape, and every kernel processes all problems of a call at once
// (grid.y, or the transform index of the FFT engine), so the launch count of a batched solve equals
// that of a single solve.
#pragma once
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/tikh.h"
#include "common.cuh"
#include "fft.cuh"

namespace tikh {

constexpr int MAX_DEPTH = 40;

// one basis matrix B(z) per problem: 25 polynomials (entry (i,j) at c + pb*cstride + (5i+j)*cap),
// device-side lengths (32 per problem) and per-column max |Re|,|Im| bit patterns (8 per problem)
// that fix the lazy power-of-two column scaling
struct BasisBuf {
  cd* c = nullptr;
  int* len = nullptr;
  unsigned long long* colmax = nullptr;
  int64_t cap = 0;
  __host__ __device__ int64_t cstride() const { return 25 * cap; }
  __device__ cd* cp(int pb) const { return c + pb * cstride(); }
  __device__ int* lp(int pb) const { return len + pb * 32; }
  __device__ unsigned long long* mp(int pb) const { return colmax + pb * 8; }
};

// DFS schedule of Algorithm 1: a node (a, s, L) at `depth` has nodes omega^{a + c + s j}, c in {0,1},
// j < L (s L = N) and 4L conditions.
enum StepKind { STEP_LEAF = 0, STEP_EVAL = 1, STEP_PROD = 2 };
constexpr int BATCH_PROD_DIRECT_MAX = 36;  // automatic thresholds for plans with batch > 1 (measured)
constexpr int BATCH_EVAL_DIRECT_MAX = 10;

struct Step {
  int kind;
  int depth;
  int side;  // 0: left child (writes buf[depth][0]), 1: right child
  int64_t a, s, L;
  int fft;          // FFT plan index: eval length L/2 (STEP_EVAL) or product length P (STEP_PROD)
  int64_t P;        // product transform length (STEP_PROD)
  uint64_t save_mask;  // STEP_LEAF: depths whose delta_in is this leaf's delta_in
};

// per-problem user arrays of a call: element i of problem pb at base + pb * stride + i
struct UserArrays {
  const void* col = nullptr;
  const void* row = nullptr;
  const void* rhs = nullptr;
  void* x = nullptr;
  int64_t col_stride = 0, row_stride = 0, rhs_stride = 0, x_stride = 0;
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
  int batch_max = 1;
  int nb = 1;          // problems in the current call
  int slack_mult = 1;  // degree-prediction slack multiplier (raised after TIKH_EDEGREE)
  int64_t eval_direct_max = 80;   // step 2 by direct evaluation when the right child has <= this many nodes per coset
  int64_t prod_direct_max = 360;  // step 4 by schoolbook products when the planned length P <= this
  int wait_polls = 1 << 24;       // bounded wait of the leaf's rebuild warps (polls)

  std::vector<Step> sched;
  std::map<int64_t, int> fft_of_len;
  std::vector<FftPlan> ffts;
  std::map<int64_t, cd*> twiddle_of_len;
  int64_t Pmax = 0, Lrmax = 0;

  // device memory (per-problem arrays: leading problem index)
  std::vector<void*> allocs;
  int64_t bytes = 0;
  cd* wN = nullptr;     // omega^e, e < N (shared)
  cd* specT = nullptr;  // [nb][N] DFT of the circulant generator of the core T
  cd* work = nullptr;   // [nb][N]
  cd* work2 = nullptr;  // [nb][N]
  cd* ftmpN = nullptr;  // [nb][N] four-step temp for length-N transforms
  cd* R = nullptr;      // [nb][N][2][5] residual rows
  cd* Phi = nullptr;    // [nb][N][2][5] original condition rows
  int* delta = nullptr;   // [nb][8]
  int* dstack = nullptr;  // [nb][MAX_DEPTH][5]
  int* status = nullptr;  // 1 (shared by the batch)
  int* ndiff = nullptr;   // [nb][4]
  int* bad = nullptr;     // [nb] 1: non-finite input (set by the prologue's check)
  int64_t* diff = nullptr;  // [nb][max_difficult] condition ids 2e + f
  cd* diffr = nullptr;      // [nb][max_difficult][5] residuals
  cd* dvals = nullptr;      // [nb][max_difficult][25] B*(sigma) of the deferred conditions
  BasisBuf buf[MAX_DEPTH][2];
  cd* evalv = nullptr;  // [nb][50][Lrmax]
  cd* etmp = nullptr;   // [nb][50][Lrmax] (four-step temp)
  cd* FA = nullptr;     // [nb][25][Pmax] spectra of B_L
  cd* FB = nullptr;     // [nb][25][Pmax] spectra of B_R
  cd* FC = nullptr;     // [nb][25][Pmax] products
  cd* ptmp = nullptr;   // [nb][50][Pmax] (four-step temp)
  unsigned long long* peak = nullptr;  // [nb] fill magnitude (bit pattern of a non-negative double)
  double* lam = nullptr;  // [nb] regularisation weights of the current call
  cd* ybuf = nullptr;    // [nb][cn] core right-hand side
  cd* rbuf = nullptr;    // [nb][cn] refinement residual
  cd* xcore = nullptr;   // [nb][cn] core solution
  cd* dx = nullptr;      // [nb][cn] refinement correction
  double* norms = nullptr;  // [nb][4]: ||r||^2, ||y||^2 of the last residual
  cd* dscr = nullptr;    // [nb][dscr_stride] difficult-point scratch
  int64_t dscr_stride = 0;
  void* d_in = nullptr;  // staging for tikh_solve_host: col | row | b | x
  cd* gbuf = nullptr;    // [nb][4N + 2cm] adjoint workspace (first gradient call)
  double* gdl = nullptr; // [nb] dL/dlambda
  int64_t launches = 0;

  // optional CUDA graph of the whole solve, replayed while the call's arguments stay the same
  cudaGraphExec_t graph_exec = nullptr;
  UserArrays graph_key{};
  int graph_nb = 0, graph_rhs_is_y = -1;

  // optional timing of every leaf launch with a CUDA event pair on the plan's stream
  int prof_leaf = 0;  // profiling flags (bit 0: leaves, bit 1: every launch group by kind)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<signed char> ev_kind;  // kind of each recorded pair (-1: a leaf timed for bit 0 only)
  size_t ev_used = 0;

  tikh_stats last{};
};

// launchers (return the number of kernels enqueued, or a negative TIKH_E* code)
int launch_twiddle(cd* tab, int64_t L, cudaStream_t s);
int launch_spectrum(Plan& P, const UserArrays& u, int rhs_is_y);
int launch_rhs(Plan& P, const UserArrays& u, int rhs_is_y);
int launch_conditions(Plan& P, const cd* y);
int launch_extract(Plan& P, cd* out);
int launch_residual(Plan& P, const cd* y, const cd* x, cd* r);
int launch_axpy(Plan& P, cd* x, const cd* dx);
int launch_output(Plan& P, const cd* v, const UserArrays& u);
int launch_leaf(Plan& P, const Step& st);
int launch_eval(Plan& P, const Step& st);
int launch_prod(Plan& P, const Step& st);
int launch_difficult(Plan& P);
int launch_grad(Plan& P, const void* x, int64_t x_stride, const void* b, int64_t b_stride, void* dcol,
                int64_t dcol_stride, void* drow, int64_t drow_stride, void* db, int64_t db_stride, double* dlam,
                cd* gbuf);
int launch_leaf_arrays(int K, const cd* sigma, const cd* r, int* delta, double eps, cd* B, int* len,
                       unsigned long long* colmax, int* ndiff, int64_t* diff, int* status, int* order, int* pivot,
                       cudaStream_t s);
int launch_fft_test(int64_t L, cd* data, int sign, cudaStream_t s, int64_t* bytes_out);

}  // namespace tikh
