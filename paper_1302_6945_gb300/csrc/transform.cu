// transform.cu -- extension and transformation (Sec. 3.1, 3.3, 4.1), extraction (Sec. 5) and the
// FFT matrix-vector products used by refinement (cf. Sec. 7.3).
//
// The core problem is tall (cm >= cn): (T^H T + lam I) x = y.  For m < n the core matrix is T^H
// (a'_d = conj(a_{-d})) and its right-hand side is b itself; the answer is then x = T^H v.
//
// Conditions at node e (omega = exp(+2 pi i / N)):
//   F_e = [lam omega^{e(cm+k-1)}, lamH_e, 1, 0, yhat_e],  G_e = [-that_e, omega^{e(cn+k-1)}, 0, 1, 0]
// with that = DFT(c_T), c_T[j] = a_{j-(cn+k-1)} over the N-periodic extended sequence,
// lamH_e = omega^{e(k-1)} conj(that_e) (the T^H generator's DFT, obtained in O(N) as in Sec. 7.3),
// yhat = DFT of -y placed after cm+k-1 zeros.
//
// Length-N transforms run one transform per problem (transform index = problem index).
#include "internal.h"

namespace tikh {

// ------------------------------------------------------------------------------------------------
__global__ void k_twiddle(cd* tab, int64_t L) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < L; t += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)t / (double)L, &s, &c);
    tab[t] = mkc(c, s);
  }
}

int launch_twiddle(cd* tab, int64_t L, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((L + 255) / 256, 4096);
  k_twiddle<<<blocks, 256, 0, s>>>(tab, L);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// user data access
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ cd load_user(const void* p, int64_t i, int dtype) {
  if (dtype == TIKH_C128) return ((const cd*)p)[i];
  return mkc(((const double*)p)[i], 0.0);
}
__device__ __forceinline__ void store_user(void* p, int64_t i, int dtype, cd v) {
  if (dtype == TIKH_C128) ((cd*)p)[i] = v;
  else ((double*)p)[i] = v.x;
}

// diagonal d of problem pb's core matrix (d in [-(cn-1), cm-1])
struct CoreDiag {
  const void* col;
  const void* row;
  int64_t col_stride, row_stride;
  int dtype, dual;
  __device__ cd operator()(int pb, int64_t d) const {
    int64_t oc = pb * col_stride, orow = pb * row_stride;
    if (!dual) return d >= 0 ? load_user(col, oc + d, dtype) : load_user(row, orow - d, dtype);
    // a'_d = conj(a_{-d})
    cd v = d <= 0 ? load_user(col, oc - d, dtype) : load_user(row, orow + d, dtype);
    return cconj(v);
  }
};

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based hash, mapped to [-1, 1)
__device__ __forceinline__ double splitmix_uniform(unsigned long long c) {
  unsigned long long z = 0x5eedULL + (c + 1ULL) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// peak = max over the known diagonals of max(|Re|, |Im|)  (exact, order independent); and the input
// check: a non-finite diagonal or right-hand-side entry marks the problem (bad[pb] = 1, whose leaves
// then process no condition) and the call (ST_INPUT), so no kernel iterates on NaN or Inf
__global__ void k_peak(CoreDiag a, int64_t cm, int64_t cn, unsigned long long* peak, const void* rhs,
                       int64_t rhs_stride, int64_t rhs_len, int dtype, int* bad, int* status) {
  const int pb = blockIdx.y;
  double mx = 0.0;
  bool fin = true;
  int64_t total = cm + cn - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = a(pb, i - (cn - 1));
    fin = fin && isfinite(v.x) && isfinite(v.y);
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rhs_len; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = load_user(rhs, pb * rhs_stride + i, dtype);
    fin = fin && isfinite(v.x) && isfinite(v.y);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(peak + pb, (unsigned long long)__double_as_longlong(mx));
  if (!fin) {
    bad[pb] = 1;
    set_status(status, ST_INPUT);
  }
}

// c_T[j] = a_{j-(cn+k-1)} over the periodic sequence; entries a_{cm-1+i}, i = 1..k, are the fill
struct LoadGenerator {
  CoreDiag a;
  int64_t cm, cn, N, k;
  int fill, is_complex;
  const unsigned long long* peak;
  __device__ cd operator()(int pb, int64_t j) const {
    int64_t d = ((j - (cn + k - 1)) % N + N) % N;
    if (d <= cm - 1) return a(pb, d);
    if (d >= N - (cn - 1)) return a(pb, d - N);
    int64_t i = d - (cm - 1);  // 1..k
    if (fill == 1) {
      cd lo = a(pb, -(cn - 1)), hi = a(pb, cm - 1);
      double f = (double)i / (double)(k + 1);
      return mkc(hi.x + (lo.x - hi.x) * f, hi.y + (lo.y - hi.y) * f);
    }
    double pk = __longlong_as_double((long long)peak[pb]);
    double re = pk * splitmix_uniform((unsigned long long)(2 * i));
    double im = is_complex ? pk * splitmix_uniform((unsigned long long)(2 * i + 1)) : 0.0;
    return mkc(re, im);
  }
};
// plain per-problem vectors: element j of problem pb at base + pb * stride + j
struct StoreVec {
  cd* out;
  int64_t stride;
  __device__ void operator()(int pb, int64_t k, cd v) const { out[pb * stride + k] = v; }
};
struct LoadVec {
  const cd* in;
  int64_t stride;
  __device__ cd operator()(int pb, int64_t j) const { return in[pb * stride + j]; }
};
// [v; 0]: user vector of length len, zero beyond
struct LoadPadUser {
  const void* v;
  int64_t stride, len;
  int dtype;
  __device__ cd operator()(int pb, int64_t j) const {
    return j < len ? load_user(v, pb * stride + j, dtype) : mkc(0.0, 0.0);
  }
};
// [v; 0]: complex vector of length len, zero beyond
struct LoadPadC {
  const cd* v;
  int64_t stride, len;
  __device__ cd operator()(int pb, int64_t j) const { return j < len ? v[pb * stride + j] : mkc(0.0, 0.0); }
};
// spectrum times lamH_e = omega^{e(k-1)} conj(that_e)  (adjoint generator, Sec. 7.3)
struct StoreMulLamH {
  cd* out;
  const cd* that;
  const cd* wN;
  int64_t N, k;
  __device__ void operator()(int pb, int64_t e, cd v) const {
    int64_t t = ((e * (k - 1)) % N + N) % N;
    out[pb * N + e] = cmul(v, cmul(tw_at(wN, t), cconj(that[pb * N + e])));
  }
};
struct StoreMulT {
  cd* out;
  const cd* that;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd v) const { out[pb * N + e] = cmul(v, that[pb * N + e]); }
};
// window [off, off + len) of an inverse transform, scaled, into a compact vector
struct StoreWindowC {
  cd* out;
  int64_t stride, off, len;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    if (j >= off && j < off + len) out[pb * stride + j - off] = cscale(v, scale);
  }
};
// window of the inverse transform [off, off+len) scaled by 1/N into the user output
struct StoreWindowUser {
  void* out;
  int64_t stride, off, len;
  int dtype;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    if (j >= off && j < off + len) store_user(out, pb * stride + j - off, dtype, cscale(v, scale));
  }
};
// -y (complex, length len) placed at offset off
struct LoadPlaceNegC {
  const cd* y;
  int64_t stride, off, len;
  __device__ cd operator()(int pb, int64_t j) const {
    if (j < off || j >= off + len) return mkc(0.0, 0.0);
    cd v = y[pb * stride + j - off];
    return mkc(-v.x, -v.y);
  }
};
// conditions F_e, G_e into R and Phi
struct StoreConditions {
  cd* R;
  cd* Phi;
  const cd* that;
  const cd* wN;
  const double* lam;
  int64_t N, cm, cn, k;
  __device__ void operator()(int pb, int64_t e, cd yh) const {
    cd th = that[pb * N + e];
    cd wF = tw_at(wN, (e * (cm + k - 1)) % N);
    cd wG = tw_at(wN, (e * (cn + k - 1)) % N);
    cd lh = cmul(tw_at(wN, ((e * (k - 1)) % N + N) % N), cconj(th));
    cd row[10] = {cscale(wF, lam[pb]), lh, mkc(1.0, 0.0), mkc(0.0, 0.0), yh,
                  mkc(-th.x, -th.y), wG, mkc(0.0, 0.0), mkc(1.0, 0.0), mkc(0.0, 0.0)};
    int64_t base = (pb * N + e) * 10;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      R[base + i] = row[i];
      Phi[base + i] = row[i];
    }
  }
};

__global__ void k_reset_peak(unsigned long long* peak, int* bad, int nb) {
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    peak[i] = 0ULL;
    bad[i] = 0;
  }
}
__global__ void k_reset_tree(int* delta, int d0, int d1, int d2, int d3, int* ndiff, int nb) {
  for (int pb = threadIdx.x; pb < nb; pb += blockDim.x) {
    int* d = delta + 8 * pb;
    d[0] = d0; d[1] = d1; d[2] = d2; d[3] = d3; d[4] = 0;
    ndiff[4 * pb] = 0;
  }
}

static inline dim3 grid2(int64_t n, int nb, int threads = 256, int cap = 4096) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap)), (unsigned)nb);
}

// that = DFT(c_T) of each problem's core matrix (Sec. 3.1, Eq. (circdiag))
int launch_spectrum(Plan& P, const UserArrays& u, int rhs_is_y) {
  cudaStream_t s = P.stream;
  int nl = 0, r;
  k_reset_peak<<<1, 256, 0, s>>>(P.peak, P.bad, P.nb);
  ++nl;
  CoreDiag a{u.col, u.row, u.col_stride, u.row_stride, P.dtype, P.dual};
  // the user right-hand side: y (n entries) for the normal-equation form, else b (m entries)
  const int64_t rhs_len = rhs_is_y ? P.n : P.m;
  k_peak<<<grid2(P.cm + P.cn, P.nb, 256, 1024), 256, 0, s>>>(a, P.cm, P.cn, P.peak, u.rhs, u.rhs_stride, rhs_len,
                                                              P.dtype, P.bad, P.status);
  ++nl;
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  const FftPlan& FN = P.ffts[P.fft_of_len.at(P.N)];
  LoadGenerator lg{a, P.cm, P.cn, P.N, P.k, P.opts.fill, P.dtype == TIKH_C128 ? 1 : 0, P.peak};
  if ((r = fft_run(FN, P.nb, +1, lg, StoreVec{P.specT, P.N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  return nl + r;
}

__global__ void k_to_complex(const void* in, int64_t stride, int dtype, int64_t n, cd* out) {
  const int pb = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[pb * n + i] = load_user(in, pb * stride + i, dtype);
}

// core right-hand side y (complex, cn per problem): T^H b, or the given vector (user y, or b for m < n)
int launch_rhs(Plan& P, const UserArrays& u, int rhs_is_y) {
  cudaStream_t s = P.stream;
  int nl = 0, r;
  const int64_t N = P.N, k = P.k, cm = P.cm, cn = P.cn;
  if (rhs_is_y) {
    k_to_complex<<<grid2(cn, P.nb), 256, 0, s>>>(u.rhs, u.rhs_stride, P.dtype, cn, P.ybuf);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  // y = T^H b: rows cm+k-1.. of circ(c_H) [b; 0] (Sec. 3.1), DFT(c_H) = lamH
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  if ((r = fft_run(FN, P.nb, +1, LoadPadUser{u.rhs, u.rhs_stride, cm, P.dtype},
                   StoreMulLamH{P.work, P.specT, P.wN, N, k}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, StoreWindowC{P.ybuf, cn, cm + k - 1, cn, 1.0 / (double)N},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  return nl + r;
}

// conditions F, G of the core system with right-hand side y (Sec. 3.3, 4.1); resets the degrees
int launch_conditions(Plan& P, const cd* y) {
  cudaStream_t s = P.stream;
  const int64_t N = P.N, k = P.k, cm = P.cm, cn = P.cn;
  // Eq. (taudef) with tau = [cn-1, cm-1, cm+k-2, cn+k-2, 0]; the starting basis has delta = -tau
  k_reset_tree<<<1, 256, 0, s>>>(P.delta, -(int)(cn - 1), -(int)(cm - 1), -(int)(cm + k - 2), -(int)(cn + k - 2),
                                 P.ndiff, P.nb);
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  StoreConditions sc{P.R, P.Phi, P.specT, P.wN, P.lam, N, cm, cn, k};
  int r = fft_run(FN, P.nb, +1, LoadPlaceNegC{y, cn, cm + k - 1, cn}, sc, P.ftmpN, s);
  if (r < 0) return TIKH_ECUDA;
  return r + 1;
}

// ------------------------------------------------------------------------------------------------
// extraction: x(z) = B*_1^{(j)}(z) / B*_5^{(j)}, j the column of tau-degree 0 (Sec. 4.3 end, 5)
// ------------------------------------------------------------------------------------------------
__global__ void k_extract(BasisBuf B, const int* delta, int* status, int64_t cn, cd* out) {
  const int pb = blockIdx.y;
  const int* dl = delta + 8 * pb;
  int js = -1, nz = 0, no = 0;
  for (int j = 0; j < 5; ++j) {
    int d = dl[j];
    if (d == 0) { js = j; ++nz; } else if (d == 1) ++no;
  }
  bool ok = nz == 1 && no == 4;
  cd c5 = mkc(0.0, 0.0);
  const cd* c = B.cp(pb);
  const int* len = B.lp(pb);
  if (ok) {
    if (len[20 + js] >= 1) c5 = c[(int64_t)(20 + js) * B.cap];
    ok = cnonzero(c5);
  }
  if (!ok) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, ST_NUMERIC);
    return;
  }
  double den = cabs2(c5);
  cd inv = mkc(c5.x / den, -c5.y / den);
  const cd* b1 = c + (int64_t)js * B.cap;
  int64_t l1 = len[js];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cn; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = i < l1 ? cmul(b1[i], inv) : mkc(0.0, 0.0);
    if (!isfinite(v.x) || !isfinite(v.y)) set_status(status, ST_NUMERIC);
    out[pb * cn + i] = v;
  }
}

int launch_extract(Plan& P, cd* out) {
  k_extract<<<grid2(P.cn, P.nb, 256, 2048), 256, 0, P.stream>>>(P.buf[0][0], P.delta, P.status, P.cn, out);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// refinement pieces: r = y - (T_c^H T_c x + lam x) by FFT matvecs (cf. Sec. 7.3), x += dx
// ------------------------------------------------------------------------------------------------
// keep the inverse-transform window [off, N) scaled at its own index, zero before
struct StoreKeepFrom {
  cd* out;
  int64_t N, off;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    out[pb * N + j] = j >= off ? cscale(v, scale) : mkc(0.0, 0.0);
  }
};
// [u; 0] with u = in[off .. off + len)
struct LoadShift {
  const cd* in;
  int64_t N, off, len;
  __device__ cd operator()(int pb, int64_t j) const { return j < len ? in[pb * N + off + j] : mkc(0.0, 0.0); }
};
struct StoreResidual {
  cd* r;
  const cd* y;
  const cd* x;
  const double* lam;
  int64_t cn, off;
  double scale;
  double* norms;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    if (j < off || j >= off + cn) return;
    int64_t i = pb * cn + j - off;
    double l = lam[pb];
    cd ax = mkc(v.x * scale + l * x[i].x, v.y * scale + l * x[i].y);
    cd ri = csub(y[i], ax);
    r[i] = ri;
    atomicAdd(norms + 4 * pb, cabs2(ri));
    atomicAdd(norms + 4 * pb + 1, cabs2(y[i]));
  }
};

__global__ void k_zero_norms(double* p, int nb) {
  for (int i = threadIdx.x; i < 4 * nb; i += blockDim.x) p[i] = 0.0;
}

int launch_residual(Plan& P, const cd* y, const cd* x, cd* r) {
  cudaStream_t s = P.stream;
  const int64_t N = P.N, k = P.k, cm = P.cm, cn = P.cn;
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  int nl = 0, q;
  k_zero_norms<<<1, 256, 0, s>>>(P.norms, P.nb);
  ++nl;
  // u = T_c x: rows cn+k-1.. of circ(c_T) [x; 0]
  if ((q = fft_run(FN, P.nb, +1, LoadPadC{x, cn, cn}, StoreMulT{P.work, P.specT, N}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, StoreKeepFrom{P.work2, N, cn + k - 1, 1.0 / (double)N}, P.ftmpN,
                   s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  // T_c^H u: rows cm+k-1.. of circ(c_H) [u; 0]
  if ((q = fft_run(FN, P.nb, +1, LoadShift{P.work2, N, cn + k - 1, cm}, StoreMulLamH{P.work, P.specT, P.wN, N, k},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  StoreResidual sr{r, y, x, P.lam, cn, cm + k - 1, 1.0 / (double)N, P.norms};
  if ((q = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, sr, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  return nl + q;
}

__global__ void k_axpy(cd* x, const cd* dx, int64_t n) {
  const int64_t off = (int64_t)blockIdx.y * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[off + i] = cadd(x[off + i], dx[off + i]);
}

int launch_axpy(Plan& P, cd* x, const cd* dx) {
  k_axpy<<<grid2(P.cn, P.nb), 256, 0, P.stream>>>(x, dx, P.cn);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

__global__ void k_from_complex(const cd* in, int64_t n, void* out, int64_t stride, int dtype) {
  const int pb = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    store_user(out, pb * stride + i, dtype, in[pb * n + i]);
}

// user x from the core solution: x itself, or x = T^H v = T_c v for m < n
int launch_output(Plan& P, const cd* v, const UserArrays& u) {
  cudaStream_t s = P.stream;
  if (!P.dual) {
    k_from_complex<<<grid2(P.cn, P.nb), 256, 0, s>>>(v, P.cn, u.x, u.x_stride, P.dtype);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  const FftPlan& FN = P.ffts[P.fft_of_len.at(P.N)];
  int nl = 0, r;
  if ((r = fft_run(FN, P.nb, +1, LoadPadC{v, P.cn, P.cn}, StoreMulT{P.work, P.specT, P.N}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(FN, P.nb, -1, LoadVec{P.work, P.N},
                   StoreWindowUser{u.x, u.x_stride, P.cn + P.k - 1, P.cm, P.dtype, 1.0 / (double)P.N}, P.ftmpN, s)) <
      0)
    return TIKH_ECUDA;
  return nl + r;
}

}  // namespace tikh
