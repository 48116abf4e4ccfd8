// grad.cu -- hand-written adjoint of x = (T^H T + lam I)^{-1} T^H b (m >= n).
//
// With A = T^H T + lam I (Hermitian), an upstream gradient G = dL/dx (conjugate-Wirtinger
// convention of PyTorch: dL = Re(G^H dx)) and g = A^{-1} G (one more superfast solve whose
// right-hand side is G itself, Sec. 7.1's form):
//   dL/db      = T g                                     (x is linear in b, adjoint T A^{-1})
//   dL/dlambda = -Re(g^H x)                              (dx/dlambda = -A^{-1} x)
//   dL/da_d    = sum_j r_{j+d} conj(g_j) - u_{j+d} conj(x_j),  r = b - T x, u = T g
// (dx = A^{-1}(dT^H r - T^H dT x); a_d is the d-th diagonal, d in [-(n-1), m-1]).  The two
// cross-correlations are one inverse DFT of R conj(Ghat) - U conj(Xhat), all of length N >= m+n-1.
// dL/dcol[d] = dL/da_d (d >= 0), dL/drow[d] = dL/da_{-d} (d >= 1), dL/drow[0] = 0 (a_0 is col[0]).
// Real data take real parts.
#include "internal.h"

namespace tikh {

__device__ __forceinline__ cd load_user_g(const void* p, int64_t i, int dtype) {
  if (dtype == TIKH_C128) return ((const cd*)p)[i];
  return mkc(((const double*)p)[i], 0.0);
}
__device__ __forceinline__ void store_user_g(void* p, int64_t i, int dtype, cd v) {
  if (dtype == TIKH_C128) ((cd*)p)[i] = v;
  else ((double*)p)[i] = v.x;
}

struct GLoadPadUser {  // [v; 0] from a user array
  const void* v;
  int64_t stride, len;
  int dtype;
  __device__ cd operator()(int pb, int64_t j) const {
    return j < len ? load_user_g(v, pb * stride + j, dtype) : mkc(0.0, 0.0);
  }
};
struct GLoadPadC {  // [v; 0] from a complex buffer
  const cd* v;
  int64_t stride, len;
  __device__ cd operator()(int pb, int64_t j) const { return j < len ? v[pb * stride + j] : mkc(0.0, 0.0); }
};
struct GStoreVec {
  cd* out;
  int64_t N;
  __device__ void operator()(int pb, int64_t k, cd v) const { out[pb * N + k] = v; }
};
struct GLoadMulT {  // that .* spec
  const cd* that;
  const cd* spec;
  int64_t N;
  __device__ cd operator()(int pb, int64_t e) const { return cmul(that[pb * N + e], spec[pb * N + e]); }
};
// T x window (rows n+k-1 .. of the circulant product) -> r = b - T x (complex buffer)
struct GStoreResid {
  cd* r;
  const void* b;
  int64_t b_stride, off, m;
  int dtype;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    if (j < off || j >= off + m) return;
    int64_t i = j - off;
    r[pb * m + i] = csub(load_user_g(b, pb * b_stride + i, dtype), cscale(v, scale));
  }
};
// T g window -> u (complex buffer) and dL/db
struct GStoreTg {
  cd* u;
  void* db;
  int64_t db_stride, off, m;
  int dtype;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    if (j < off || j >= off + m) return;
    int64_t i = j - off;
    cd w = cscale(v, scale);
    u[pb * m + i] = w;
    store_user_g(db, pb * db_stride + i, dtype, w);
  }
};
struct GLoadCorr {  // Rhat conj(Ghat) - Uhat conj(Xhat)
  const cd* R;
  const cd* G;
  const cd* U;
  const cd* X;
  int64_t N;
  __device__ cd operator()(int pb, int64_t e) const {
    int64_t i = pb * N + e;
    return csub(cmul(R[i], cconj(G[i])), cmul(U[i], cconj(X[i])));
  }
};
struct GStoreGen {  // circular correlation index d mod N -> dL/dcol, dL/drow
  void* dcol;
  void* drow;
  int64_t col_stride, row_stride, m, n, N;
  int dtype;
  double scale;
  __device__ void operator()(int pb, int64_t t, cd v) const {
    cd w = cscale(v, scale);
    if (t < m) store_user_g(dcol, pb * col_stride + t, dtype, w);
    if (t > N - n) store_user_g(drow, pb * row_stride + (N - t), dtype, w);
    if (t == 0) store_user_g(drow, pb * row_stride, dtype, mkc(0.0, 0.0));
  }
};

// dL/dlambda = -Re(g^H x), one block per problem
__global__ void k_grad_lambda(const cd* g, const void* x, int64_t x_stride, int dtype, int64_t n, double* out) {
  __shared__ double red[32];
  const int pb = blockIdx.x;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    cd gj = g[pb * n + j], xj = load_user_g(x, pb * x_stride + j, dtype);
    acc += gj.x * xj.x + gj.y * xj.y;  // Re(conj(g) x)
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[pb] = -s;
  }
}

// the adjoint step after g (= P.xcore) is known; gbuf holds 4N + 2m complex per problem
int launch_grad(Plan& P, const void* x, int64_t x_stride, const void* b, int64_t b_stride, void* dcol,
                int64_t dcol_stride, void* drow, int64_t drow_stride, void* db, int64_t db_stride, double* dlam,
                cd* gbuf) {
  cudaStream_t s = P.stream;
  const int64_t N = P.N, k = P.k, m = P.cm, n = P.cn;
  const int nb = P.nb;
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  cd* Xh = gbuf;
  cd* Gh = Xh + (size_t)nb * N;
  cd* Rh = Gh + (size_t)nb * N;
  cd* Uh = Rh + (size_t)nb * N;
  cd* rr = Uh + (size_t)nb * N;
  cd* uu = rr + (size_t)nb * m;
  const double invN = 1.0 / (double)N;
  int nl = 0, q;
  if ((q = fft_run(FN, nb, +1, GLoadPadUser{x, x_stride, n, P.dtype}, GStoreVec{Xh, N}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, nb, +1, GLoadPadC{P.xcore, n, n}, GStoreVec{Gh, N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  nl += q;
  // r = b - T x and u = T g: rows n+k-1 .. of circ(c_T) [v; 0] (Sec. 3.1)
  if ((q = fft_run(FN, nb, -1, GLoadMulT{P.specT, Xh, N}, GStoreResid{rr, b, b_stride, n + k - 1, m, P.dtype, invN},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, nb, -1, GLoadMulT{P.specT, Gh, N}, GStoreTg{uu, db, db_stride, n + k - 1, m, P.dtype, invN},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, nb, +1, GLoadPadC{rr, m, m}, GStoreVec{Rh, N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, nb, +1, GLoadPadC{uu, m, m}, GStoreVec{Uh, N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, nb, -1, GLoadCorr{Rh, Gh, Uh, Xh, N},
                   GStoreGen{dcol, drow, dcol_stride, drow_stride, m, n, N, P.dtype, invN}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  k_grad_lambda<<<nb, 256, 0, s>>>(P.xcore, x, x_stride, P.dtype, n, dlam);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return nl + 1;
}

}  // namespace tikh
