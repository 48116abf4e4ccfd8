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
// General problem (Sec. 3.2, reading: all three block rows extended to the same N): unknowns
// [x (n), sigma_1 (m), sigma_2 (pl), gamma_1 (N-n), gamma_2 (N-m), gamma_3 (N-pl), 1] and
//   F_e = [0, lamH_e, lamLH_e, 1, 0, 0, yhat_e],  G_e = [-that_e, omega^{e(N-m)}, 0, 0, 1, 0, 0],
//   H_e = [-lhat_e, 0, omega^{e(N-pl)}, 0, 0, 1, 0]
// with lhat the DFT of L's generator (extension kl = N - (pl + n - 1)) and lamLH_e = omega^{e(kl-1)} conj(lhat_e).
//
// Length-N transforms run one transform per item (transform index = item index pb).  Every size that
// belongs to a problem (m, n, cm, cn, k) and its user arrays are read from the item table
// (ItemDev[pb]), so one launch serves items of different shapes that share N; per-item buffers of
// length cn (y, x, residual, correction) use the plan's largest cn as their stride.
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

__global__ void k_to_cf(const cd* __restrict__ in, cf* out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = to_cf(in[t]);
}

// complex64 copy of a complex128 table (each entry rounded to nearest)
int launch_to_cf(const cd* in, cf* out, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_to_cf<<<blocks, 256, 0, s>>>(in, out, n);
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

// diagonal d of an item's core matrix (d in [-(cn-1), cm-1])
__device__ __forceinline__ cd core_diag(const ItemDev& it, int64_t d, int dtype) {
  if (!it.dual) return d >= 0 ? load_user(it.col, d, dtype) : load_user(it.row, -d, dtype);
  // a'_d = conj(a_{-d})
  cd v = d <= 0 ? load_user(it.col, -d, dtype) : load_user(it.row, d, dtype);
  return cconj(v);
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based hash, mapped to [-1, 1)
__device__ __forceinline__ double splitmix_uniform(unsigned long long c) {
  unsigned long long z = 0x5eedULL + (c + 1ULL) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// peak = max over the known diagonals of max(|Re|, |Im|)  (exact, order independent); and the input
// check: a non-finite diagonal or right-hand-side entry marks the item (bad[pb] = 1, whose leaves then
// process no condition) and the call (ST_INPUT), so no kernel iterates on NaN or Inf
// diagonal d of an item's regulariser L (general plans; d in [-(n-1), pl-1])
__device__ __forceinline__ cd l_diag(const ItemDev& it, int64_t d, int dtype) {
  return d >= 0 ? load_user(it.lcol, d, dtype) : load_user(it.lrow, -d, dtype);
}

__global__ void k_peak(const ItemDev* __restrict__ items, int dtype, int rhs_is_y, unsigned long long* peak, int* bad,
                       int* status, unsigned long long* peakG, unsigned long long* peakL) {
  const int pb = blockIdx.y;
  const ItemDev it = items[pb];
  double mx = 0.0;
  bool fin = true;
  const int64_t total = it.cm + it.cn - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = core_diag(it, i - (it.cn - 1), dtype);
    fin = fin && isfinite(v.x) && isfinite(v.y);
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  // the user right-hand side: y (n entries) for the normal-equation form, else b (m entries)
  const int64_t rhs_len = rhs_is_y ? it.n : it.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rhs_len; i += (int64_t)gridDim.x * blockDim.x) {
    cd v = load_user(it.rhs, i, dtype);
    fin = fin && isfinite(v.x) && isfinite(v.y);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(peak + pb, (unsigned long long)__double_as_longlong(mx));
  if (it.gram) {  // Toeplitz-Gramian: G's first column (n entries), its own fill magnitude
    double mg = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.cn; i += (int64_t)gridDim.x * blockDim.x) {
      cd v = load_user(it.gram, i, dtype);
      fin = fin && isfinite(v.x) && isfinite(v.y);
      mg = fmax(mg, fmax(fabs(v.x), fabs(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mg = fmax(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    if ((threadIdx.x & 31) == 0 && mg > 0.0) atomicMax(peakG + pb, (unsigned long long)__double_as_longlong(mg));
  }
  if (it.lcol) {  // general problem: L's diagonals, its own fill magnitude
    double ml = 0.0;
    const int64_t tl = it.pl + it.cn - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tl; i += (int64_t)gridDim.x * blockDim.x) {
      cd v = l_diag(it, i - (it.cn - 1), dtype);
      fin = fin && isfinite(v.x) && isfinite(v.y);
      ml = fmax(ml, fmax(fabs(v.x), fabs(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) ml = fmax(ml, __shfl_xor_sync(0xffffffffu, ml, o));
    if ((threadIdx.x & 31) == 0 && ml > 0.0) atomicMax(peakL + pb, (unsigned long long)__double_as_longlong(ml));
  }
  if (!fin) {
    bad[pb] = 1;
    set_status(status, ST_INPUT);
  }
}

// c_T[j] = a_{j-(cn+k-1)} over the periodic sequence; entries a_{cm-1+i}, i = 1..k, are the fill
struct LoadGenerator {
  const ItemDev* items;
  int64_t N;
  int fill, dtype;
  const unsigned long long* peak;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    const int64_t cm = it.cm, cn = it.cn, k = it.k;
    int64_t d = ((j - (cn + k - 1)) % N + N) % N;
    if (d <= cm - 1) return core_diag(it, d, dtype);
    if (d >= N - (cn - 1)) return core_diag(it, d - N, dtype);
    int64_t i = d - (cm - 1);  // 1..k
    if (fill == 1) {
      cd lo = core_diag(it, -(cn - 1), dtype), hi = core_diag(it, cm - 1, dtype);
      double f = (double)i / (double)(k + 1);
      return mkc(hi.x + (lo.x - hi.x) * f, hi.y + (lo.y - hi.y) * f);
    }
    double pk = __longlong_as_double((long long)peak[pb]);
    double re = pk * splitmix_uniform((unsigned long long)(2 * i));
    double im = dtype == TIKH_C128 ? pk * splitmix_uniform((unsigned long long)(2 * i + 1)) : 0.0;
    return mkc(re, im);
  }
};
// general plans: c_L[j] = l_{j-(n+kl-1)} over L's N-periodic sequence; the kl entries l_{pl-1+i} are the
// fill, as T's (R5) but from L's own peak and with counters offset by 2^41
struct LoadLGenerator {
  const ItemDev* items;
  int64_t N;
  int fill, dtype;
  const unsigned long long* peakL;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    const int64_t pl = it.pl, n = it.cn, kl = it.kl;
    int64_t d = ((j - (n + kl - 1)) % N + N) % N;
    if (d <= pl - 1) return l_diag(it, d, dtype);
    if (d >= N - (n - 1)) return l_diag(it, d - N, dtype);
    int64_t i = d - (pl - 1);  // 1..kl
    if (fill == 1) {
      cd lo = l_diag(it, -(n - 1), dtype), hi = l_diag(it, pl - 1, dtype);
      double f = (double)i / (double)(kl + 1);
      return mkc(hi.x + (lo.x - hi.x) * f, hi.y + (lo.y - hi.y) * f);
    }
    const double pk = __longlong_as_double((long long)peakL[pb]);
    const unsigned long long off = 1ULL << 41;
    const double re = pk * splitmix_uniform((unsigned long long)(2 * i) + off);
    const double im = dtype == TIKH_C128 ? pk * splitmix_uniform((unsigned long long)(2 * i + 1) + off) : 0.0;
    return mkc(re, im);
  }
};
// Toeplitz-Gramian (Sec. 3.4, Eq. (gramblk)): the x-column of the first block row is the n x n Hermitian
// Toeplitz G below N - n extension rows, whose circulant generator is c11[(N - n + d) mod N] = g_d for
// |d| <= n - 1 (g_{-d} = conj(g_d)); the N - 2n + 1 other entries are the extension's arbitrary entries,
// filled like L's (R5) with counters offset by 2^40 (fill = 1: a linear ramp from g_{n-1} to conj(g_{n-1}))
struct LoadGramGenerator {
  const ItemDev* items;
  int64_t N;
  int fill, dtype;
  const unsigned long long* peakG;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    const int64_t n = it.cn;
    const int64_t d = ((j - (N - n)) % N + N) % N;
    if (d <= n - 1) return load_user(it.gram, d, dtype);
    if (d >= N - (n - 1)) return cconj(load_user(it.gram, N - d, dtype));
    const int64_t i = d - (n - 1), nfill = N - 2 * n + 1;  // 1 .. nfill
    if (fill == 1) {
      const cd hi = load_user(it.gram, n - 1, dtype), lo = cconj(hi);
      const double f = (double)i / (double)(nfill + 1);
      return mkc(hi.x + (lo.x - hi.x) * f, hi.y + (lo.y - hi.y) * f);
    }
    const double pk = __longlong_as_double((long long)peakG[pb]);
    const unsigned long long off = 1ULL << 40;
    const double re = pk * splitmix_uniform((unsigned long long)(2 * i) + off);
    const double im = dtype == TIKH_C128 ? pk * splitmix_uniform((unsigned long long)(2 * i + 1) + off) : 0.0;
    return mkc(re, im);
  }
};
// plain per-item vectors: element j of item pb at base + pb * stride + j
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
// [b; 0]: the item's user right-hand side b (cm entries), zero beyond
struct LoadPadUserRhs {
  const ItemDev* items;
  int dtype;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    return j < it.cm ? load_user(it.rhs, j, dtype) : mkc(0.0, 0.0);
  }
};
// [v; 0]: the item's complex vector of length cn (stride = the plan's largest cn), zero beyond
struct LoadPadCn {
  const cd* v;
  const ItemDev* items;
  int64_t stride;
  __device__ cd operator()(int pb, int64_t j) const { return j < items[pb].cn ? v[pb * stride + j] : mkc(0.0, 0.0); }
};
// spectrum times lamH_e = omega^{e(k-1)} conj(that_e)  (adjoint generator, Sec. 7.3)
struct StoreMulLamH {
  cd* out;
  const cd* that;
  const cd* wN;
  const ItemDev* items;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd v) const {
    const int64_t k = items[pb].k;
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
// window [cm + k - 1, cm + k - 1 + cn) of an inverse transform, scaled, into the item's y
struct StoreWindowY {
  cd* out;
  const ItemDev* items;
  int64_t stride;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    const ItemDev& it = items[pb];
    const int64_t off = it.cm + it.k - 1;
    if (j >= off && j < off + it.cn) out[pb * stride + j - off] = cscale(v, scale);
  }
};
// window [cn + k - 1, cn + k - 1 + cm) of the inverse transform, scaled by 1/N, into the user x (m < n)
struct StoreWindowUserX {
  const ItemDev* items;
  int dtype;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    const ItemDev& it = items[pb];
    const int64_t off = it.cn + it.k - 1;
    if (j >= off && j < off + it.cm) store_user(it.x, j - off, dtype, cscale(v, scale));
  }
};
// -y (the item's cn entries) placed at offset cm + k - 1
struct LoadPlaceNegY {
  const cd* y;
  const ItemDev* items;
  int64_t stride;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    const int64_t off = it.cm + it.k - 1;
    if (j < off || j >= off + it.cn) return mkc(0.0, 0.0);
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
  const ItemDev* items;
  const cd* specG;  // Toeplitz-Gramian plans: DFT of G's generator (F's x component); null for l2
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd yh) const {
    const ItemDev& it = items[pb];
    const int64_t cm = it.cm, cn = it.cn, k = it.k;
    cd th = that[pb * N + e];
    cd wF = tw_at(wN, (e * (cm + k - 1)) % N);
    cd wG = tw_at(wN, (e * (cn + k - 1)) % N);
    cd lh = cmul(tw_at(wN, ((e * (k - 1)) % N + N) % N), cconj(th));
    const cd f0 = specG ? specG[pb * N + e] : cscale(wF, lam[pb]);
    cd row[10] = {f0, lh, mkc(1.0, 0.0), mkc(0.0, 0.0), yh,
                  mkc(-th.x, -th.y), wG, mkc(0.0, 0.0), mkc(1.0, 0.0), mkc(0.0, 0.0)};
    int64_t base = (pb * N + e) * 10;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
      R[base + i] = row[i];
      Phi[base + i] = row[i];
    }
  }
};

// conditions F_e, G_e, H_e of the general problem into R and Phi (21 entries per node)
struct StoreConditionsGeneral {
  cd* R;
  cd* Phi;
  const cd* that;
  const cd* lhat;
  const cd* wN;
  const ItemDev* items;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd yh) const {
    const ItemDev& it = items[pb];
    const int64_t m = it.cm, n = it.cn, pl = it.pl, k = it.k, kl = it.kl;
    const cd th = that[pb * N + e], lh = lhat[pb * N + e];
    const cd tH = cmul(tw_at(wN, ((e * (k - 1)) % N + N) % N), cconj(th));
    const cd lH = cmul(tw_at(wN, ((e * (kl - 1)) % N + N) % N), cconj(lh));
    const cd wG = tw_at(wN, (e * (N - m)) % N), wH = tw_at(wN, (e * (N - pl)) % N);
    const cd z = mkc(0.0, 0.0), one = mkc(1.0, 0.0);
    (void)n;
    cd row[21] = {z, tH, lH, one, z, z, yh,
                  mkc(-th.x, -th.y), wG, z, z, one, z, z,
                  mkc(-lh.x, -lh.y), z, wH, z, z, one, z};
    const int64_t base = (pb * N + e) * 21;
#pragma unroll
    for (int i = 0; i < 21; ++i) {
      R[base + i] = row[i];
      Phi[base + i] = row[i];
    }
  }
};

__global__ void k_reset_peak(unsigned long long* peak, int* bad, unsigned long long* peakG, unsigned long long* peakL,
                             int nb) {
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    peak[i] = 0ULL;
    bad[i] = 0;
    if (peakG) peakG[i] = 0ULL;
    if (peakL) peakL[i] = 0ULL;
  }
}
// Eq. (taudef) with tau = [cn-1, cm-1, cm+k-2, cn+k-2, 0] (reading R3), or for the general problem
// tau = [n-1, m-1, pl-1, N-n-1, N-m-1, N-pl-1, 0] (tau_i + 1 = the length of unknown i); the starting
// basis I has tau-degrees delta = -tau
__global__ void k_reset_tree(const ItemDev* __restrict__ items, int* delta, int* ndiff, int nb, int general,
                             int64_t N) {
  for (int pb = threadIdx.x; pb < nb; pb += blockDim.x) {
    const ItemDev& it = items[pb];
    int* d = delta + DSTR * pb;
    if (general) {
      d[0] = -(int)(it.cn - 1);
      d[1] = -(int)(it.cm - 1);
      d[2] = -(int)(it.pl - 1);
      d[3] = -(int)(N - it.cn - 1);
      d[4] = -(int)(N - it.cm - 1);
      d[5] = -(int)(N - it.pl - 1);
      d[6] = 0;
    } else {
      d[0] = -(int)(it.cn - 1);
      d[1] = -(int)(it.cm - 1);
      d[2] = -(int)(it.cm + it.k - 2);
      d[3] = -(int)(it.cn + it.k - 2);
      d[4] = 0;
    }
    ndiff[4 * pb] = 0;
  }
}

static inline dim3 grid2(int64_t n, int nb, int threads = 256, int cap = 4096) {
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap)), (unsigned)nb);
}

// that = DFT(c_T) of each item's core matrix (Sec. 3.1, Eq. (circdiag)), after the input check
int launch_spectrum(Plan& P, int rhs_is_y) {
  cudaStream_t s = P.stream;
  int nl = 0, r;
  k_reset_peak<<<1, 256, 0, s>>>(P.peak, P.bad, P.peakG, P.peakL, P.nb);
  ++nl;
  k_peak<<<grid2(std::max(std::max(P.cm + P.cn, P.m), P.pl + P.cn), P.nb, 256, 1024), 256, 0, s>>>(
      P.items, P.dtype, rhs_is_y, P.peak, P.bad, P.status, P.peakG, P.peakL);
  ++nl;
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  const FftPlan& FN = P.ffts[P.fft_of_len.at(P.N)];
  LoadGenerator lg{P.items, P.N, P.opts.fill, P.dtype, P.peak};
  if ((r = fft_run(FN, P.nb, +1, lg, StoreVec{P.specT, P.N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  nl += r;
  if (P.gram) {  // DFT of G's circulant generator (F's x component, Sec. 3.4)
    LoadGramGenerator lgg{P.items, P.N, P.opts.fill, P.dtype, P.peakG};
    if ((r = fft_run(FN, P.nb, +1, lgg, StoreVec{P.specG, P.N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
    nl += r;
  }
  if (P.general) {  // DFT of L's circulant generator (Sec. 3.2)
    LoadLGenerator llg{P.items, P.N, P.opts.fill, P.dtype, P.peakL};
    if ((r = fft_run(FN, P.nb, +1, llg, StoreVec{P.specL, P.N}, P.ftmpN, s)) < 0) return TIKH_ECUDA;
    nl += r;
  }
  return nl;
}

// the item's user vector (cn entries: y, or b for m < n) as complex, stride = the plan's largest cn
__global__ void k_rhs_to_complex(const ItemDev* __restrict__ items, int dtype, int64_t stride, cd* out) {
  const int pb = blockIdx.y;
  const ItemDev it = items[pb];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.cn; i += (int64_t)gridDim.x * blockDim.x)
    out[pb * stride + i] = load_user(it.rhs, i, dtype);
}

// core right-hand side y (complex, cn per item): T^H b, or the given vector (user y, or b for m < n)
int launch_rhs(Plan& P, int rhs_is_y) {
  cudaStream_t s = P.stream;
  int nl = 0, r;
  const int64_t N = P.N;
  if (rhs_is_y) {
    k_rhs_to_complex<<<grid2(P.cn, P.nb), 256, 0, s>>>(P.items, P.dtype, P.cn, P.ybuf);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  // y = T^H b: rows cm+k-1.. of circ(c_H) [b; 0] (Sec. 3.1), DFT(c_H) = lamH
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  if ((r = fft_run(FN, P.nb, +1, LoadPadUserRhs{P.items, P.dtype}, StoreMulLamH{P.work, P.specT, P.wN, P.items, N},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, StoreWindowY{P.ybuf, P.items, P.cn, 1.0 / (double)N}, P.ftmpN,
                   s)) < 0)
    return TIKH_ECUDA;
  return nl + r;
}

// conditions F, G (and H for the general problem) of the core system with right-hand side y (Sec. 3.2,
// 3.3, 4.1); resets the degrees
int launch_conditions(Plan& P, const cd* y) {
  cudaStream_t s = P.stream;
  const int64_t N = P.N;
  k_reset_tree<<<1, 256, 0, s>>>(P.items, P.delta, P.ndiff, P.nb, P.general, N);
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  int r;
  if (P.general) {
    StoreConditionsGeneral sc{P.R, P.Phi, P.specT, P.specL, P.wN, P.items, N};
    r = fft_run(FN, P.nb, +1, LoadPlaceNegY{y, P.items, P.cn}, sc, P.ftmpN, s);
  } else {
    StoreConditions sc{P.R, P.Phi, P.specT, P.wN, P.lam, P.items, P.gram ? P.specG : nullptr, N};
    r = fft_run(FN, P.nb, +1, LoadPlaceNegY{y, P.items, P.cn}, sc, P.ftmpN, s);
  }
  if (r < 0) return TIKH_ECUDA;
  return r + 1;
}

// ------------------------------------------------------------------------------------------------
// extraction: x(z) = B*_1^{(j)}(z) / B*_W^{(j)}, j the column of tau-degree 0 (Sec. 4.3 end, 5)
// ------------------------------------------------------------------------------------------------
template <int W>
__global__ void k_extract(BasisBuf B, const int* delta, int* status, const ItemDev* __restrict__ items, int64_t stride,
                          cd* out) {
  const int pb = blockIdx.y;
  const int64_t cn = items[pb].cn;
  const int* dl = delta + DSTR * pb;
  int js = -1, nz = 0, no = 0;
  for (int j = 0; j < W; ++j) {
    int d = dl[j];
    if (d == 0) { js = j; ++nz; } else if (d == 1) ++no;
  }
  bool ok = nz == 1 && no == W - 1;
  cd c5 = mkc(0.0, 0.0);
  const cd* c = B.cp(pb);
  const int* len = B.lp(pb);
  if (ok) {
    const int last = W * (W - 1) + js;
    if (len[last] >= 1) c5 = c[(int64_t)last * B.cap];
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
    out[pb * stride + i] = v;
  }
}

int launch_extract(Plan& P, cd* out) {
  if (P.w == 7)
    k_extract<7><<<grid2(P.cn, P.nb, 256, 2048), 256, 0, P.stream>>>(P.buf[0][0], P.delta, P.status, P.items, P.cn, out);
  else
    k_extract<5><<<grid2(P.cn, P.nb, 256, 2048), 256, 0, P.stream>>>(P.buf[0][0], P.delta, P.status, P.items, P.cn, out);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// refinement pieces: r = y - (T_c^H T_c x + lam x) by FFT matvecs (cf. Sec. 7.3), x += dx
// ------------------------------------------------------------------------------------------------
// keep the inverse-transform window [cn + k - 1, N) scaled at its own index, zero before
struct StoreKeepFrom {
  cd* out;
  const ItemDev* items;
  int64_t N;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    const int64_t off = items[pb].cn + items[pb].k - 1;
    out[pb * N + j] = j >= off ? cscale(v, scale) : mkc(0.0, 0.0);
  }
};
// [u; 0] with u = in[cn + k - 1 .. cn + k - 1 + cm)
struct LoadShift {
  const cd* in;
  const ItemDev* items;
  int64_t N;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    return j < it.cm ? in[pb * N + it.cn + it.k - 1 + j] : mkc(0.0, 0.0);
  }
};
struct StoreResidual {
  cd* r;
  const cd* y;
  const cd* x;
  const double* lam;
  const ItemDev* items;
  int64_t stride;
  double scale;
  double* norms;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    const ItemDev& it = items[pb];
    const int64_t off = it.cm + it.k - 1;
    if (j < off || j >= off + it.cn) return;
    int64_t i = pb * stride + j - off;
    double l = lam[pb];
    cd ax = mkc(v.x * scale + l * x[i].x, v.y * scale + l * x[i].y);
    cd ri = csub(y[i], ax);
    r[i] = ri;
    atomicAdd(norms + 4 * pb, cabs2(ri));
    atomicAdd(norms + 4 * pb + 1, cabs2(y[i]));
  }
};

// norms[4 pb + 0, 1]: ||r||^2, ||y||^2 of the last residual; [4 pb + 2, 3]: ||dx||^2, ||x + dx||^2 of the
// last correction.  k_zero_norms clears the pair starting at `first` (0 or 2) of every item.
__global__ void k_zero_norms(double* p, int nb, int first) {
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    p[4 * i + first] = 0.0;
    p[4 * i + first + 1] = 0.0;
  }
}

// T_c^H u spectrum (lamH U) plus, for Toeplitz-Gramian plans, G's spectrum times X = DFT([x; 0]): the inverse
// transform's window [N - n, N) is then L^H L x + G x
struct StoreMulLamHPlusG {
  cd* out;
  const cd* that;
  const cd* wN;
  const ItemDev* items;
  const cd* specG;
  const cd* X;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd v) const {
    const int64_t k = items[pb].k;
    int64_t t = ((e * (k - 1)) % N + N) % N;
    const int64_t i = pb * N + e;
    out[i] = cfma(specG[i], X[i], cmul(v, cmul(tw_at(wN, t), cconj(that[i]))));
  }
};
// stores t_hat X and X itself (the refinement of a Toeplitz-Gramian plan needs both)
struct StoreMulTKeep {
  cd* out;
  cd* keep;
  const cd* that;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd v) const {
    out[pb * N + e] = cmul(v, that[pb * N + e]);
    keep[pb * N + e] = v;
  }
};

// general plans: X = DFT([x; 0]) (kept in gX) times L's spectrum, inverse, keep the window of L x
struct LoadMulSpec {
  const cd* X;
  const cd* spec;
  int64_t N;
  __device__ cd operator()(int pb, int64_t j) const { return cmul(X[pb * N + j], spec[pb * N + j]); }
};
// keep the inverse-transform window [n + kl - 1, N) (L x) scaled at its own index, zero before
struct StoreKeepFromL {
  cd* out;
  const ItemDev* items;
  int64_t N;
  double scale;
  __device__ void operator()(int pb, int64_t j, cd v) const {
    const int64_t off = items[pb].cn + items[pb].kl - 1;
    out[pb * N + j] = j >= off ? cscale(v, scale) : mkc(0.0, 0.0);
  }
};
// [w; 0] with w = in[n + kl - 1 .. n + kl - 1 + pl) (L x)
struct LoadShiftL {
  const cd* in;
  const ItemDev* items;
  int64_t N;
  __device__ cd operator()(int pb, int64_t j) const {
    const ItemDev& it = items[pb];
    return j < it.pl ? in[pb * N + it.cn + it.kl - 1 + j] : mkc(0.0, 0.0);
  }
};
// out += spectrum times lamLH_e = omega^{e(kl-1)} conj(lhat_e)  (L^H applied in the transform domain)
struct StoreAddMulLamLH {
  cd* out;
  const cd* lhat;
  const cd* wN;
  const ItemDev* items;
  int64_t N;
  __device__ void operator()(int pb, int64_t e, cd v) const {
    const int64_t kl = items[pb].kl;
    const int64_t t = ((e * (kl - 1)) % N + N) % N;
    const int64_t i = pb * N + e;
    out[i] = cfma(v, cmul(tw_at(wN, t), cconj(lhat[i])), out[i]);
  }
};

int launch_residual(Plan& P, const cd* y, const cd* x, cd* r) {
  cudaStream_t s = P.stream;
  const int64_t N = P.N;
  const FftPlan& FN = P.ffts[P.fft_of_len.at(N)];
  int nl = 0, q;
  k_zero_norms<<<1, 256, 0, s>>>(P.norms, P.nb, 0);
  ++nl;
  // u = T_c x: rows cn+k-1.. of circ(c_T) [x; 0]
  if (P.gram || P.general)
    q = fft_run(FN, P.nb, +1, LoadPadCn{x, P.items, P.cn}, StoreMulTKeep{P.work, P.gX, P.specT, N}, P.ftmpN, s);
  else
    q = fft_run(FN, P.nb, +1, LoadPadCn{x, P.items, P.cn}, StoreMulT{P.work, P.specT, N}, P.ftmpN, s);
  if (q < 0) return TIKH_ECUDA;
  nl += q;
  if ((q = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, StoreKeepFrom{P.work2, P.items, N, 1.0 / (double)N}, P.ftmpN,
                   s)) < 0)
    return TIKH_ECUDA;
  nl += q;
  // T_c^H u: rows cm+k-1.. of circ(c_H) [u; 0] (plus G x for Toeplitz-Gramian plans, same rows)
  if (P.gram)
    q = fft_run(FN, P.nb, +1, LoadShift{P.work2, P.items, N},
                StoreMulLamHPlusG{P.work, P.specT, P.wN, P.items, P.specG, P.gX, N}, P.ftmpN, s);
  else
    q = fft_run(FN, P.nb, +1, LoadShift{P.work2, P.items, N}, StoreMulLamH{P.work, P.specT, P.wN, P.items, N},
                P.ftmpN, s);
  if (q < 0) return TIKH_ECUDA;
  nl += q;
  if (P.general) {  // + L^H L x: rows n+kl-1.. of circ(c_L) [x; 0], then L^H by lamLH, added to T^H T x
    if ((q = fft_run(FN, P.nb, -1, LoadMulSpec{P.gX, P.specL, N}, StoreKeepFromL{P.work2, P.items, N, 1.0 / (double)N},
                     P.ftmpN, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
    if ((q = fft_run(FN, P.nb, +1, LoadShiftL{P.work2, P.items, N}, StoreAddMulLamLH{P.work, P.specL, P.wN, P.items, N},
                     P.ftmpN, s)) < 0)
      return TIKH_ECUDA;
    nl += q;
  }
  StoreResidual sr{r, y, x, P.lam, P.items, P.cn, 1.0 / (double)N, P.norms};
  if ((q = fft_run(FN, P.nb, -1, LoadVec{P.work, N}, sr, P.ftmpN, s)) < 0) return TIKH_ECUDA;
  return nl + q;
}

__global__ void k_axpy(cd* x, const cd* dx, const ItemDev* __restrict__ items, int64_t stride, double* norms) {
  __shared__ double red[2][8];
  const int64_t off = (int64_t)blockIdx.y * stride, n = items[blockIdx.y].cn;
  double sd = 0.0, sx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cd d = dx[off + i], v = cadd(x[off + i], d);
    x[off + i] = v;
    sd += cabs2(d);
    sx += cabs2(v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sd; red[1][threadIdx.x >> 5] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { sd += red[0][w]; sx += red[1][w]; }
    atomicAdd(norms + 4 * blockIdx.y + 2, sd);
    atomicAdd(norms + 4 * blockIdx.y + 3, sx);
  }
}

// x += dx, accumulating ||dx||^2 and ||x + dx||^2 (the relative size of the last correction)
int launch_axpy(Plan& P, cd* x, const cd* dx) {
  k_zero_norms<<<1, 256, 0, P.stream>>>(P.norms, P.nb, 2);
  k_axpy<<<grid2(P.cn, P.nb), 256, 0, P.stream>>>(x, dx, P.items, P.cn, P.norms);
  return cudaGetLastError() == cudaSuccess ? 2 : TIKH_ECUDA;
}

__global__ void k_output_direct(const cd* in, int64_t stride, const ItemDev* __restrict__ items, int dtype) {
  const int pb = blockIdx.y;
  const ItemDev it = items[pb];
  if (it.dual) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < it.cn; i += (int64_t)gridDim.x * blockDim.x)
    store_user(it.x, i, dtype, in[pb * stride + i]);
}

// user x from the core solution: x itself, or x = T^H v = T_c v for m < n (the plan's items are
// either all direct or all dual: the two forms have different core shapes)
int launch_output(Plan& P, const cd* v) {
  cudaStream_t s = P.stream;
  if (!P.dual) {
    k_output_direct<<<grid2(P.cn, P.nb), 256, 0, s>>>(v, P.cn, P.items, P.dtype);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  const FftPlan& FN = P.ffts[P.fft_of_len.at(P.N)];
  int nl = 0, r;
  if ((r = fft_run(FN, P.nb, +1, LoadPadCn{v, P.items, P.cn}, StoreMulT{P.work, P.specT, P.N}, P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(FN, P.nb, -1, LoadVec{P.work, P.N}, StoreWindowUserX{P.items, P.dtype, 1.0 / (double)P.N},
                   P.ftmpN, s)) < 0)
    return TIKH_ECUDA;
  return nl + r;
}

}  // namespace tikh
