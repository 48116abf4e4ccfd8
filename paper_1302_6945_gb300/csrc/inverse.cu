// inverse.cu -- one solver for many right-hand sides: the displacement representation of
// X = (T^H T + lam I)^{-1} (m >= n), built from eight superfast solves and applied by FFT correlations.
//
// The paper solves one right-hand side per run: b enters the conditions' fifth component and every pivot
// decision (Sec. 4.3), so one interpolation basis serves one b.  The matrix itself carries over.  With Z the
// n x n down-shift, e_0, f = e_{n-1} and t_d the diagonals of T,
//   A - Z A Z^H = p p^H - q q^H + e_0 s^H + s e_0^H,  p_j = conj(t_{-j}), q_j = conj(t_{m-j}) (q_0 = 0),
//   s = A e_0 - t_0 p  (s_0 halved; the terms below never read it),
// and multiplying Z A Z^H = A - (...) by X on both sides (Z^H Z = I - f f^H) gives X - Z^H X Z as four
// rank-one terms u_t w_t^H:
//   (u_0, w_0) = (f - Z^H X Z A f, X f),   (u_1, w_1) = (Z^H X p, X Z^H p),
//   (u_2, w_2) = (-Z^H X q, X Z^H q),       (u_3, w_3) = (Z^H X e_0, X Z^H s).
// Z is nilpotent, so the Stein equation sums to X = sum_{k<n} (Z^H)^k (X - Z^H X Z) Z^k, i.e.
//   X y = sum_t H(u_t) H(w_t)^H y,   H(u)_{ik} = u_{i+k} (0 for i + k >= n),
// two correlations per term.  All correlations and Toeplitz products run as length-N transforms of the
// FFT engine (N >= m + n - 1, the plan's circulant length, so nothing wraps):
//   with F the sign +1 DFT and F^-1 = F_{-1} / N:  F^-1(conj(F w) F v)_k = sum_j conj(w_j) v_{j+k},
//   T x  = F^-1(F a . F x) at rows n-1 .. n+m-2,  a_d = t_{d-(n-1)} (d < m + n - 1),
//   T^H v = F^-1(conj(F a) . F v) at index (j - (n-1)) mod N for output j,
//   c_t = H(w_t)^H y = F(F y . conj(W_t)) / N, kept for k < n,
//   X y = F_{-1}(sum_t F_{-1}(c_t) . U_t) / N, kept for i < n  (U_t = F u_t, W_t = F w_t).
// An apply is ten transforms per right-hand side (twelve from b, with T^H b), a refinement correction
// r = y - A x, x += X~ r fourteen more (Sec. 7.2's pattern with the FFT matvec of Sec. 7.3).
#include "internal.h"

namespace tikh {

__device__ __forceinline__ cd inv_load_user(const void* p, int64_t i, int dtype) {
  if (dtype == TIKH_C128) return ((const cd*)p)[i];
  return mkc(((const double*)p)[i], 0.0);
}
__device__ __forceinline__ void inv_store_user(void* p, int64_t i, int dtype, cd v) {
  if (dtype == TIKH_C128) ((cd*)p)[i] = v;
  else ((double*)p)[i] = v.x;
}
// t_d, d in [-(n-1), m-1]: col[d] for d >= 0, row[-d] below (row[0] is not read)
__device__ __forceinline__ cd inv_diag(const void* col, const void* row, int64_t d, int dtype) {
  return d >= 0 ? inv_load_user(col, d, dtype) : inv_load_user(row, -d, dtype);
}

// ---- loaders (transform b, index j < N) and storers (transform b, index k < N) ----

// a_d = t_{d-(n-1)} for d < m + n - 1, zero beyond
struct ILoadGen {
  const void *col, *row;
  int64_t m, n;
  int dtype;
  __device__ cd operator()(int, int64_t d) const {
    return d < m + n - 1 ? inv_diag(col, row, d - (n - 1), dtype) : mkc(0.0, 0.0);
  }
};
// transform 0: T e_0 (T's first column, col[0..m)); transform 1: T f (T's last column, a_0 .. a_{m-1})
struct ILoadColumns {
  const void *col, *row;
  int64_t m, n;
  int dtype;
  __device__ cd operator()(int b, int64_t j) const {
    if (j >= m) return mkc(0.0, 0.0);
    return b == 0 ? inv_load_user(col, j, dtype) : inv_diag(col, row, j - (n - 1), dtype);
  }
};
// [v; 0] of user vectors (length len, element stride between transforms)
struct ILoadUser {
  const void* v;
  int64_t stride, len;
  int dtype;
  __device__ cd operator()(int b, int64_t j) const {
    return j < len ? inv_load_user(v, (int64_t)b * stride + j, dtype) : mkc(0.0, 0.0);
  }
};
// [v; 0] of internal vectors (length len, rows of `stride`)
struct ILoadVec {
  const cd* v;
  int64_t stride, len;
  __device__ cd operator()(int b, int64_t j) const { return j < len ? v[(int64_t)b * stride + j] : mkc(0.0, 0.0); }
};
// spec[b] . S (S one spectrum shared by every transform), or conj(S) when `conjS`
struct ILoadMulShared {
  const cd* spec;
  const cd* S;
  int64_t N;
  int conjS;
  __device__ cd operator()(int b, int64_t e) const {
    const cd s = S[e];
    return cmul(spec[(int64_t)b * N + e], conjS ? cconj(s) : s);
  }
};
// transform bb = 4 r + t: Y_r . conj(W_t)
struct ILoadYW {
  const cd* Y;
  const cd* W;  // W_0 .. W_3, N apart
  int64_t N;
  __device__ cd operator()(int bb, int64_t e) const { return cmul(Y[(int64_t)(bb >> 2) * N + e], cconj(W[(int64_t)(bb & 3) * N + e])); }
};
// transform r: sum_t G_{4r+t}
struct ILoadSum4 {
  const cd* G;
  int64_t N;
  __device__ cd operator()(int r, int64_t e) const {
    const cd* g = G + (int64_t)4 * r * N + e;
    return cadd(cadd(g[0], g[N]), cadd(g[2 * N], g[3 * N]));
  }
};

struct IStoreVec {  // out[b][k] = v
  cd* out;
  int64_t N;
  __device__ void operator()(int b, int64_t k, cd v) const { out[(int64_t)b * N + k] = v; }
};
// c_t: out[bb][k] = v / N for k < n, zero beyond (the next transform reads the whole row)
struct IStoreTrunc {
  cd* out;
  int64_t N, n;
  double scale;
  __device__ void operator()(int bb, int64_t k, cd v) const {
    out[(int64_t)bb * N + k] = k < n ? cscale(v, scale) : mkc(0.0, 0.0);
  }
};
// out[bb][e] = v . U_{bb mod 4}
struct IStoreMulU {
  cd* out;
  const cd* U;  // U_0 .. U_3, N apart
  int64_t N;
  __device__ void operator()(int bb, int64_t e, cd v) const {
    out[(int64_t)bb * N + e] = cmul(v, U[(int64_t)(bb & 3) * N + e]);
  }
};
// x[b][i] = v / N (or += when `accumulate`) for i < n
struct IStoreHead {
  cd* x;
  int64_t n;
  double scale;
  int accumulate;
  __device__ void operator()(int b, int64_t i, cd v) const {
    if (i >= n) return;
    cd* p = x + (int64_t)b * n + i;
    const cd w = cscale(v, scale);
    *p = accumulate ? cadd(*p, w) : w;
  }
};
// T x: u[b][i] = v / N at transform index i + n - 1, i < m
struct IStoreTx {
  cd* u;
  int64_t m, n;
  double scale;
  __device__ void operator()(int b, int64_t k, cd v) const {
    const int64_t i = k - (n - 1);
    if (i >= 0 && i < m) u[(int64_t)b * m + i] = cscale(v, scale);
  }
};
// T^H v at output j = (k + n - 1) mod N, j < n.  mode 0: y = T^H v; mode 1: y = T^H v + lam e_{idx(b)}
// (idx 0 = 0, idx 1 = n - 1: A e_0 and A f); mode 2: r = y - lam x - T^H v (the residual of A x = y)
struct IStoreTH {
  cd* out;
  const cd* y;
  const cd* x;
  int64_t n, N;
  double scale, lam;
  int mode;
  __device__ void operator()(int b, int64_t k, cd v) const {
    int64_t j = k + n - 1;
    if (j >= N) j -= N;
    if (j >= n) return;
    const int64_t o = (int64_t)b * n + j;
    cd w = cscale(v, scale);
    if (mode == 1 && j == (b == 0 ? 0 : n - 1)) w.x += lam;
    if (mode == 2) {
      const cd xv = x[o], yv = y[o];
      w = mkc(yv.x - lam * xv.x - w.x, yv.y - lam * xv.y - w.y);
    }
    out[o] = w;
  }
};

// ---- elementwise kernels ----

// the eight right-hand sides v_0..v_7 = f, Z A f, p, q, e_0, Z^H p, Z^H q, Z^H s (user dtype, n apart)
__global__ void k_inv_rhs(const void* col, const void* row, int64_t m, int64_t n, int dtype, const cd* Ae,
                          void* rhs) {
  const int i = blockIdx.y;
  const cd t0 = inv_load_user(col, 0, dtype);
  auto p = [&](int64_t j) { return cconj(j == 0 ? t0 : inv_load_user(row, j, dtype)); };
  auto q = [&](int64_t j) { return j == 0 ? mkc(0.0, 0.0) : cconj(inv_load_user(col, m - j, dtype)); };
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const bool up = j + 1 < n;  // (Z^H v)_j = v_{j+1}
    cd v = mkc(0.0, 0.0);
    switch (i) {
      case 0: v = mkc(j == n - 1 ? 1.0 : 0.0, 0.0); break;
      case 1: if (j >= 1) v = Ae[n + j - 1]; break;  // Z (A f)
      case 2: v = p(j); break;
      case 3: v = q(j); break;
      case 4: v = mkc(j == 0 ? 1.0 : 0.0, 0.0); break;
      case 5: if (up) v = p(j + 1); break;
      case 6: if (up) v = q(j + 1); break;
      default:  // Z^H s, s_{j+1} = (A e_0)_{j+1} - t_0 p_{j+1}
        if (up) v = csub(Ae[j + 1], cmul(t0, p(j + 1)));
        break;
    }
    inv_store_user(rhs, (int64_t)i * n + j, dtype, v);
  }
}

// the terms from the solutions s_i = X v_i (user dtype, n apart): gen = u_0..u_3, w_0..w_3 (n apart)
__global__ void k_inv_terms(const void* sol, int64_t n, int dtype, cd* gen) {
  const int t = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const bool up = j + 1 < n;
    auto S = [&](int i, int64_t k) { return inv_load_user(sol, (int64_t)i * n + k, dtype); };
    cd v = mkc(0.0, 0.0);
    switch (t) {
      case 0: {  // f - Z^H X Z A f
        v = mkc(j == n - 1 ? 1.0 : 0.0, 0.0);
        if (up) v = csub(v, S(1, j + 1));
        break;
      }
      case 1: if (up) v = S(2, j + 1); break;                        // Z^H X p
      case 2: if (up) { const cd s = S(3, j + 1); v = mkc(-s.x, -s.y); } break;  // -Z^H X q
      case 3: if (up) v = S(4, j + 1); break;                        // Z^H X e_0
      case 4: v = S(0, j); break;                                    // X f
      case 5: v = S(5, j); break;                                    // X Z^H p
      case 6: v = S(6, j); break;                                    // X Z^H q
      default: v = S(7, j); break;                                   // X Z^H s
    }
    gen[(int64_t)t * n + j] = v;
  }
}

// user vectors (stride apart) <-> internal rows of n
__global__ void k_inv_gather(const void* src, int64_t stride, int64_t n, int dtype, cd* dst) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[(int64_t)b * n + j] = inv_load_user(src, (int64_t)b * stride + j, dtype);
}
__global__ void k_inv_scatter(const cd* src, int64_t n, int dtype, void* dst, int64_t stride) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    inv_store_user(dst, (int64_t)b * stride + j, dtype, src[(int64_t)b * n + j]);
}

static inline dim3 inv_grid(int64_t n, int rows) {
  int64_t bx = (n + 255) / 256;
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)rows);
}

// A = F a; A e_0 and A f by T^H of T's first and last columns; the eight right-hand sides
int launch_inv_prepare(const FftPlan& F, InvWork& w, const void* col, const void* row, cudaStream_t s) {
  const int64_t N = w.N;
  int nl = 0, q;
  if ((q = fft_run(F, 1, +1, ILoadGen{col, row, w.m, w.n, w.dtype}, IStoreVec{w.spec, N}, w.tmp, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(F, 2, +1, ILoadColumns{col, row, w.m, w.n, w.dtype}, IStoreVec{w.Y, N}, w.tmp, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(F, 2, -1, ILoadMulShared{w.Y, w.spec, N, 1},
                   IStoreTH{w.Ae, nullptr, nullptr, w.n, N, 1.0 / (double)N, w.lam, 1}, w.tmp, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  k_inv_rhs<<<inv_grid(w.n, 8), 256, 0, s>>>(col, row, w.m, w.n, w.dtype, w.Ae, w.rhs8);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return nl + 1;
}

// the four terms from the eight solutions, and their spectra U_t, W_t
int launch_inv_terms(const FftPlan& F, InvWork& w, cudaStream_t s) {
  k_inv_terms<<<inv_grid(w.n, 8), 256, 0, s>>>(w.sol8, w.n, w.dtype, w.gen);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  const int q = fft_run(F, 8, +1, ILoadVec{w.gen, w.n, w.n}, IStoreVec{w.spec + w.N, w.N}, w.tmp, s);
  return q < 0 ? TIKH_ECUDA : q + 1;
}

// x (rows of n) = X~ src (rows of n) for nb right-hand sides, or x += X~ src
static int inv_solve(const FftPlan& F, InvWork& w, int nb, const cd* src, cd* x, int accumulate, cudaStream_t s) {
  const int64_t N = w.N, n = w.n;
  const double sc = 1.0 / (double)N;
  int nl = 0, q;
  if ((q = fft_run(F, nb, +1, ILoadVec{src, n, n}, IStoreVec{w.Y, N}, w.tmp, s)) < 0) return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(F, 4 * nb, +1, ILoadYW{w.Y, w.spec + 5 * N, N}, IStoreTrunc{w.C, N, n, sc}, w.tmp, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(F, 4 * nb, -1, ILoadVec{w.C, N, N}, IStoreMulU{w.G, w.spec + N, N}, w.tmp, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(F, nb, -1, ILoadSum4{w.G, N}, IStoreHead{x, n, sc, accumulate}, w.tmp, s)) < 0) return TIKH_ECUDA;
  return nl + q;
}

// nb right-hand sides (user vectors `b_stride` apart: b itself, or y = T^H b when `normal`) -> x (user
// vectors `x_stride` apart), with `refine` corrections x += X~(y - A x)
int launch_inv_apply(const FftPlan& F, InvWork& w, int nb, const void* b, int64_t b_stride, int normal, int refine,
                     void* x, int64_t x_stride, cudaStream_t s) {
  if (nb < 1 || nb > w.R) return TIKH_EINVAL;
  const int64_t N = w.N, n = w.n, m = w.m;
  const double sc = 1.0 / (double)N;
  int nl = 0, q;
  if (normal) {
    k_inv_gather<<<inv_grid(n, nb), 256, 0, s>>>(b, b_stride, n, w.dtype, w.y);
    if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
    ++nl;
  } else {  // y = T^H b
    if ((q = fft_run(F, nb, +1, ILoadUser{b, b_stride, m, w.dtype}, IStoreVec{w.Y, N}, w.tmp, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
    if ((q = fft_run(F, nb, -1, ILoadMulShared{w.Y, w.spec, N, 1},
                     IStoreTH{w.y, nullptr, nullptr, n, N, sc, 0.0, 0}, w.tmp, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
  }
  if ((q = inv_solve(F, w, nb, w.y, w.x, 0, s)) < 0) return q;
  nl += q;
  for (int it = 0; it < refine; ++it) {  // r = y - lam x - T^H (T x); x += X~ r
    if ((q = fft_run(F, nb, +1, ILoadVec{w.x, n, n}, IStoreVec{w.Y, N}, w.tmp, s)) < 0) return TIKH_ECUDA;
    nl += q;
    if ((q = fft_run(F, nb, -1, ILoadMulShared{w.Y, w.spec, N, 0}, IStoreTx{w.u, m, n, sc}, w.tmp, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
    if ((q = fft_run(F, nb, +1, ILoadVec{w.u, m, m}, IStoreVec{w.Y, N}, w.tmp, s)) < 0) return TIKH_ECUDA;
    nl += q;
    if ((q = fft_run(F, nb, -1, ILoadMulShared{w.Y, w.spec, N, 1}, IStoreTH{w.r, w.y, w.x, n, N, sc, w.lam, 2},
                     w.tmp, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
    if ((q = inv_solve(F, w, nb, w.r, w.x, 1, s)) < 0) return q;
    nl += q;
  }
  k_inv_scatter<<<inv_grid(n, nb), 256, 0, s>>>(w.x, n, w.dtype, x, x_stride);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return nl + 1;
}

}  // namespace tikh
