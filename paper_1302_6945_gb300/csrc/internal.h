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
constexpr int WMAX = 7;  // largest basis size: 5 (l2, Toeplitz-Gramian), 7 (general problem, Sec. 3.2)
constexpr int DSTR = 8;  // stride of per-problem degree vectors (delta, the delta_in stack)

// one basis matrix B(z) per problem: ww = W^2 polynomials (entry (i,j) at c + pb*cstride + (W i+j)*cap),
// device-side lengths (64 per problem) and per-column max |Re|,|Im| bit patterns (8 per problem)
// that fix the lazy power-of-two column scaling
struct BasisBuf {
  cd* c = nullptr;
  int* len = nullptr;
  unsigned long long* colmax = nullptr;
  int64_t cap = 0;
  int ww = 25;
  __host__ __device__ int64_t cstride() const { return ww * cap; }
  __device__ cd* cp(int pb) const { return c + pb * cstride(); }
  __device__ int* lp(int pb) const { return len + pb * 64; }
  __device__ unsigned long long* mp(int pb) const { return colmax + pb * 8; }
};

// DFS schedule of Algorithm 1: a node (a, s, L) at `depth` has nodes omega^{a + c + s j}, c in {0,1},
// j < L (s L = N) and 2 NS L conditions (NS condition sets per node: 2, or 3 for the general problem).
enum StepKind { STEP_LEAF = 0, STEP_EVAL = 1, STEP_PROD = 2 };
// automatic direct/FFT thresholds of step 4 (product length P) and step 2 (nodes per coset) for plans with
// more than one item per launch (measured on GB300): fewer items than SMs leave the GPU room for the
// direct forms' many small blocks; at least one item per SM makes the FP64 arithmetic the bound, where the
// O(P log P) transform forms win earlier
constexpr int BATCH_PROD_DIRECT_MAX = 72, BATCH_EVAL_DIRECT_MAX = 20;            // items < SMs
constexpr int FULL_BATCH_PROD_DIRECT_MAX = 36, FULL_BATCH_EVAL_DIRECT_MAX = 10;  // items >= SMs

struct Step {
  int kind;
  int depth;
  int side;  // 0: left child (writes buf[depth][0]), 1: right child
  int64_t a, s, L;
  int fft;          // FFT plan index: eval length L/2 (STEP_EVAL) or product length P (STEP_PROD)
  int64_t P;        // product transform length (STEP_PROD)
  uint64_t save_mask;  // STEP_LEAF: depths whose delta_in is this leaf's delta_in
  // STEP_EVAL / STEP_PROD: the columns the water-filling prediction pivots in the left child (sl) and the
  // right child (sr), i.e. the rows of their bases that are not identity rows (the cost model's count)
  unsigned sl = 0u, sr = 0u;
};

// Shape of one problem: user m x n, the core (tall) problem cm x cn (cm >= cn; T^H for m < n) and the
// extension k = N - (cm + cn - 1) for the plan's N.
struct Shape {
  int64_t m = 0, n = 0, cm = 0, cn = 0, k = 0;
  int64_t pl = 0, kl = 0;  // general problem: rows of L, its extension N - (pl + n - 1)
  int dual = 0;
};

// One item of a call -- a (problem, lambda) pair -- as the kernels see it: its user arrays and shape.
// Every kernel that depends on the problem's sizes reads them here (item index = problem index pb of
// the launch), so the items of one launch may have different m, n, k as long as they share N.
struct ItemDev {
  const void* col;
  const void* row;
  const void* rhs;
  void* x;
  const void* gram;  // Toeplitz-Gramian plans: first column of the Hermitian Toeplitz G (n entries)
  const void* lcol;  // general plans: the regulariser L (pl x n), first column and first row
  const void* lrow;
  int64_t m, n, cm, cn, k;
  int64_t pl, kl;    // general plans: rows of L and its extension kl = N - (pl + n - 1)
  int dual;
  int pad_;
};

struct Plan {
  // problem
  int64_t m = 0, n = 0;
  int dtype = 0;
  tikh_opts opts{};
  cudaStream_t stream = nullptr;
  int dual = 0;
  int64_t cm = 0, cn = 0;  // core (tall) problem: cm >= cn (the largest over `shapes`)
  int64_t N = 0, M = 0, k = 0;
  std::vector<Shape> shapes;  // the shapes this plan serves (one for a single-shape plan)
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
  std::map<int64_t, cf*> twiddle32_of_len;  // complex64 copies (FP32 stages)
  int prec = TIKH_PREC_FP64;
  int gram = 0;          // 1: the Toeplitz-Gramian problem (G + L^H L) x = y (Sec. 3.4); L plays T's part
  int general = 0;       // 1: the general problem (T^H T + L^H L) x = y (Sec. 3.2)
  int w = 5, ns = 2;     // basis size and condition sets per node (7 and 3 for the general problem)
  int64_t pl = 0;        // general plans: rows of L (the largest over the shapes)
  cd* specL = nullptr;   // [nb][N] DFT of L's circulant generator (general plans)
  unsigned long long* peakL = nullptr;  // [nb] fill magnitude of L's extension
  cd* specG = nullptr;   // [nb][N] DFT of G's circulant generator (Gramian plans)
  cd* gX = nullptr;      // [nb][N] refinement scratch: DFT of [x; 0] (Gramian plans)
  unsigned long long* peakG = nullptr;  // [nb] fill magnitude of G's extension
  bool stage32 = false;  // the recursion's FFT stages in FP32 (TIKH_PREC_FP32, TIKH_PREC_FP32_REFINE)
  cf* wN32 = nullptr;    // omega^e, e < N, complex64 (FP32 evaluation folds)
  int64_t Pmax = 0, Lrmax = 0;

  // device memory (per-problem arrays: leading problem index)
  std::vector<void*> allocs;
  int64_t bytes = 0;
  cd* wN = nullptr;     // omega^e, e < N (shared)
  cd* specT = nullptr;  // [nb][N] DFT of the circulant generator of the core T
  cd* work = nullptr;   // [nb][N]
  cd* work2 = nullptr;  // [nb][N]
  cd* ftmpN = nullptr;  // [nb][N] four-step temp for length-N transforms
  cd* R = nullptr;      // [nb][N][ns][w] residual rows
  cd* Phi = nullptr;    // [nb][N][ns][w] original condition rows
  int* delta = nullptr;   // [nb][DSTR]
  int* dstack = nullptr;  // [nb][MAX_DEPTH][DSTR]
  int* status = nullptr;  // 1 (shared by the batch)
  int* ndiff = nullptr;   // [nb][4]
  int* bad = nullptr;     // [nb] 1: non-finite input (set by the prologue's check)
  int64_t* diff = nullptr;  // [nb][max_difficult] condition ids ns e + f
  cd* diffr = nullptr;      // [nb][max_difficult][w] residuals
  cd* dvals = nullptr;      // [nb][max_difficult][w^2] B*(sigma) of the deferred conditions
  BasisBuf buf[MAX_DEPTH][2];
  cd* evalv = nullptr;  // [nb][2 w^2][Lrmax]
  cd* etmp = nullptr;   // [nb][2 w^2][Lrmax] (four-step temp)
  cd* FA = nullptr;     // [nb][w^2][Pmax] spectra of B_L
  cd* FB = nullptr;     // [nb][w^2][Pmax] spectra of B_R
  cd* FC = nullptr;     // [nb][w^2][Pmax] products
  cd* ptmp = nullptr;   // [nb][2 w^2][Pmax] (four-step temp)
  unsigned long long* peak = nullptr;  // [nb] fill magnitude (bit pattern of a non-negative double)
  double* lam = nullptr;  // [nb] regularisation weights of the current call (points into lam_base)
  ItemDev* items = nullptr;  // [nb] items of the current call (points into items_base)
  double* lam_base = nullptr;
  ItemDev* items_base = nullptr;  // [item_cap] device item tables (several waves for a batch plan)
  int64_t item_cap = 0;
  bool keep_status = false;  // true: the prologue does not clear the status word (later waves of a batch)
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

  // optional CUDA graph of the whole solve, replayed for every call with the same item count (the
  // kernels read each call's arrays and sizes from the item table)
  cudaGraphExec_t graph_exec = nullptr;
  int graph_nb = 0, graph_rhs_is_y = -1;

  // optional timing of every leaf launch with a CUDA event pair on the plan's stream
  int prof_leaf = 0;  // profiling flags (bit 0: leaves, bit 1: every launch group by kind)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<signed char> ev_kind;  // kind of each recorded pair (-1: a leaf timed for bit 0 only)
  size_t ev_used = 0;

  tikh_stats last{};
};

// Device state of one displacement representation of (T^H T + lam I)^{-1} (tikh_inverse_*): the spectra
// it is applied with and the workspace of one pass over up to R right-hand sides.
struct InvWork {
  int64_t m = 0, n = 0, N = 0;
  int dtype = 0;
  double lam = 0.0;
  int R = 1;              // right-hand sides per pass
  cd* spec = nullptr;     // [9][N]: F a, U_0..U_3, W_0..W_3 (sign +1 DFTs)
  cd* gen = nullptr;      // [8][n]: u_0..u_3, w_0..w_3
  cd* Ae = nullptr;       // [2][n]: A e_0, A f
  void* rhs8 = nullptr;   // [8][n] the eight right-hand sides (plan dtype)
  void* sol8 = nullptr;   // [8][n] their solutions (plan dtype)
  cd* Y = nullptr;        // [max(R, 2)][N]
  cd* C = nullptr;        // [4R][N]
  cd* G = nullptr;        // [4R][N]
  cd* tmp = nullptr;      // [max(4R, 8)][N] four-step temporary
  cd *y = nullptr, *x = nullptr, *r = nullptr;  // [R][n]
  cd* u = nullptr;        // [R][m]
};
int launch_inv_prepare(const FftPlan& F, InvWork& w, const void* col, const void* row, cudaStream_t s);
int launch_inv_terms(const FftPlan& F, InvWork& w, cudaStream_t s);
int launch_inv_apply(const FftPlan& F, InvWork& w, int nb, const void* b, int64_t b_stride, int normal, int refine,
                     void* x, int64_t x_stride, cudaStream_t s);

// launchers (return the number of kernels enqueued, or a negative TIKH_E* code)
int launch_twiddle(cd* tab, int64_t L, cudaStream_t s);
int launch_to_cf(const cd* in, cf* out, int64_t n, cudaStream_t s);
int launch_rcp_test(const double* d, double* out, int64_t n, cudaStream_t s);
int launch_spectrum(Plan& P, int rhs_is_y);
int launch_rhs(Plan& P, int rhs_is_y);
int launch_conditions(Plan& P, const cd* y);
int launch_extract(Plan& P, cd* out);
int launch_residual(Plan& P, const cd* y, const cd* x, cd* r);
int launch_axpy(Plan& P, cd* x, const cd* dx);
int launch_output(Plan& P, const cd* v);
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
