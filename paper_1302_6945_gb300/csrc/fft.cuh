// fft.cuh -- batched mixed-radix Stockham FFT (radices 2, 3, 4, 5, 7, 8) in shared memory, in FP64
// (complex128) or FP32 (complex64): the element type the loader returns selects the precision.
//
// Transform:  X_k = sum_j x_j exp(sign 2 pi i j k / L).  sign = +1 evaluates a polynomial with
// coefficients x at the L-th roots of unity omega_k = exp(+2 pi i k / L) (Sec. 4.1, Eq. (vandprod));
// sign = -1 is the unnormalised inverse.
//
// Each CTA holds `tb` transforms of length L <= FFT_TILE_MAX in shared memory (element j of transform
// t at sm[j * tb + t]) and runs all Stockham stages there; loads and stores go through functors so
// that packing, twisting, folding, pointwise products and trimming fuse into the transform.  Longer
// transforms use the four-step split L = L1 * L2: a column pass (L2 * batch transforms of length L1,
// inter-pass twiddles applied on store) and a row pass (L1 * batch transforms of length L2), both with
// the transform index as the contiguous dimension so global accesses coalesce.
#pragma once
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"

namespace tikh {

constexpr int FFT_TILE_MAX = 4096;
constexpr int FFT_MAX_STAGES = 24;

struct FftDesc {
  int L;
  int nst;
  unsigned char rad[FFT_MAX_STAGES];
  const cd* tw;    // tw[t] = exp(+2 pi i t / L), t < L
  const cf* tw32;  // the same table rounded to complex64 (FP32 transforms; null when not needed)
};

struct FftPlan {
  int64_t L = 0;
  int tile = 256;  // elements per CTA for transforms shorter than this (several transforms per CTA)
  bool four = false;
  int64_t L1 = 0, L2 = 0;
  FftDesc d1{}, d2{};
  const cd* twL = nullptr;    // table of length L (four-step inter-pass twiddles)
  const cf* twL32 = nullptr;  // its complex64 copy
};

// the twiddle tables of a transform in the transform's own precision
template <class C> struct Tw;
template <> struct Tw<cd> {
  static __host__ __device__ const cd* of(const FftDesc& d) { return d.tw; }
  static __host__ __device__ const cd* inter(const FftPlan& p) { return p.twL; }
};
template <> struct Tw<cf> {
  static __host__ __device__ const cf* of(const FftDesc& d) { return d.tw32; }
  static __host__ __device__ const cf* inter(const FftPlan& p) { return p.twL32; }
};

// ---------------------------------------------------------------------------------------------
// in-register DFTs of size R, for complex128 (cd) and complex64 (cf) values
// ---------------------------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ C mul_i(C a, int sign) {
  C r;
  if (sign > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
template <class C, class T>
__device__ __forceinline__ C cmk(T x, T y) {
  C r;
  r.x = x;
  r.y = y;
  return r;
}

template <int R> struct Dft;

template <> struct Dft<2> {
  template <class C> __device__ __forceinline__ static void run(C* v, int) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <> struct Dft<3> {
  template <class C> __device__ __forceinline__ static void run(C* v, int sign) {
    using T = decltype(v[0].x);
    const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
    C a = v[0], t1 = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C t2 = cmk<C>(a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y);
    C t3 = mul_i(cmk<C>(h * d.x, h * d.y), sign);
    v[0] = cadd(a, t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  }
};

template <> struct Dft<4> {
  template <class C> __device__ __forceinline__ static void run(C* v, int sign) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = mul_i(csub(v[1], v[3]), sign);
    v[0] = cadd(t0, t2);
    v[1] = cadd(t1, t3);
    v[2] = csub(t0, t2);
    v[3] = csub(t1, t3);
  }
};

template <> struct Dft<5> {
  template <class C> __device__ __forceinline__ static void run(C* v, int sign) {
    using T = decltype(v[0].x);
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
    C a = v[0];
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C p1 = cmk<C>(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
    C p2 = cmk<C>(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
    C q1 = mul_i(cmk<C>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y), sign);
    C q2 = mul_i(cmk<C>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y), sign);
    v[0] = cadd(a, cadd(t1, t2));
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
  }
};

template <> struct Dft<7> {
  template <class C> __device__ __forceinline__ static void run(C* v, int sign) {
    // pairs (v_j, v_{7-j}): X_k = a + sum_j [cos(2 pi jk/7) (v_j + v_{7-j}) + i sign sin(2 pi jk/7) (v_j - v_{7-j})]
    using T = decltype(v[0].x);
    const T c1 = (T)0.62348980185873353053, c2 = (T)-0.22252093395631440429, c3 = (T)-0.90096886790241912624;
    const T s1 = (T)0.78183148246802980871, s2 = (T)0.97492791218182360702, s3 = (T)0.43388373911755812048;
    C a = v[0];
    C t1 = cadd(v[1], v[6]), t2 = cadd(v[2], v[5]), t3 = cadd(v[3], v[4]);
    C d1 = csub(v[1], v[6]), d2 = csub(v[2], v[5]), d3 = csub(v[3], v[4]);
    C p1 = cmk<C>(a.x + c1 * t1.x + c2 * t2.x + c3 * t3.x, a.y + c1 * t1.y + c2 * t2.y + c3 * t3.y);
    C p2 = cmk<C>(a.x + c2 * t1.x + c3 * t2.x + c1 * t3.x, a.y + c2 * t1.y + c3 * t2.y + c1 * t3.y);
    C p3 = cmk<C>(a.x + c3 * t1.x + c1 * t2.x + c2 * t3.x, a.y + c3 * t1.y + c1 * t2.y + c2 * t3.y);
    // sin(2 pi jk / 7) for k = 1: (s1, s2, s3); k = 2: (s2, -s3, -s1); k = 3: (s3, -s1, s2)
    C q1 = mul_i(cmk<C>(s1 * d1.x + s2 * d2.x + s3 * d3.x, s1 * d1.y + s2 * d2.y + s3 * d3.y), sign);
    C q2 = mul_i(cmk<C>(s2 * d1.x - s3 * d2.x - s1 * d3.x, s2 * d1.y - s3 * d2.y - s1 * d3.y), sign);
    C q3 = mul_i(cmk<C>(s3 * d1.x - s1 * d2.x + s2 * d3.x, s3 * d1.y - s1 * d2.y + s2 * d3.y), sign);
    v[0] = cadd(a, cadd(t1, cadd(t2, t3)));
    v[1] = cadd(p1, q1);
    v[6] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[5] = csub(p2, q2);
    v[3] = cadd(p3, q3);
    v[4] = csub(p3, q3);
  }
};

template <> struct Dft<8> {
  template <class C> __device__ __forceinline__ static void run(C* v, int sign) {
    using T = decltype(v[0].x);
    const T r = (T)0.70710678118654752440;  // 1 / sqrt(2)
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4>::run(e, sign);
    Dft<4>::run(o, sign);
    // w8^k = exp(sign 2 pi i k / 8)
    C w1 = cmk<C>(r, (T)sign * r), w3 = cmk<C>(-r, (T)sign * r);
    C o1 = cmul(o[1], w1), o2 = mul_i(o[2], sign), o3 = cmul(o[3], w3);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// ---------------------------------------------------------------------------------------------
// one Stockham stage of radix R on tb interleaved transforms of length L; Ns = product of the
// radices already applied.  Requires blockDim.x * ceil(8 / R) * R >= tb * L.
// ---------------------------------------------------------------------------------------------
template <int R, class C>
__device__ __forceinline__ void stockham_stage(C* sm, int L, int tb, int Ns, const C* __restrict__ tw, int sign) {
  constexpr int MAXB = (8 + R - 1) / R;
  const int nb = L / R;
  const int total = nb * tb;
  const int tstride = L / (Ns * R);
  C v[MAXB][R];
#pragma unroll
  for (int c = 0; c < MAXB; ++c) {
    int g = threadIdx.x + c * blockDim.x;
    if (g < total) {
      int t = g % tb, j = g / tb, k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = sm[(j + r * nb) * tb + t];
        if (r > 0 && k > 0) {
          C w = tw_at(tw, (int64_t)(r * k) * tstride);
          if (sign < 0) w.y = -w.y;
          x = cmul(x, w);
        }
        v[c][r] = x;
      }
      Dft<R>::run(v[c], sign);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < MAXB; ++c) {
    int g = threadIdx.x + c * blockDim.x;
    if (g < total) {
      int t = g % tb, j = g / tb, k = j % Ns;
      int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[(base + r * Ns) * tb + t] = v[c][r];
    }
  }
  __syncthreads();
}

template <class C>
__device__ __forceinline__ void fft_smem(C* sm, const FftDesc& d, int tb, int sign) {
  const C* tw = Tw<C>::of(d);
  int Ns = 1;
  for (int s = 0; s < d.nst; ++s) {
    switch (d.rad[s]) {
      case 2: stockham_stage<2>(sm, d.L, tb, Ns, tw, sign); break;
      case 3: stockham_stage<3>(sm, d.L, tb, Ns, tw, sign); break;
      case 4: stockham_stage<4>(sm, d.L, tb, Ns, tw, sign); break;
      case 5: stockham_stage<5>(sm, d.L, tb, Ns, tw, sign); break;
      case 7: stockham_stage<7>(sm, d.L, tb, Ns, tw, sign); break;
      default: stockham_stage<8>(sm, d.L, tb, Ns, tw, sign); break;
    }
    Ns *= d.rad[s];
  }
}

// the element type a loader returns (cd or cf) fixes the precision of the transform
template <class LD>
using ElemOf = typename std::decay<decltype(std::declval<LD>()(0, (int64_t)0))>::type;

// A loader or storer may declare `bool active(int t)`: transform t is then computed only if both of them
// call it active (a CTA whose transforms are all inactive returns at once and writes nothing).
template <class T, class = void>
struct HasActive : std::false_type {};
template <class T>
struct HasActive<T, std::void_t<decltype(std::declval<const T&>().active(0))>> : std::true_type {};
template <class T>
__device__ __forceinline__ bool active_of(const T& f, int t) {
  if constexpr (HasActive<T>::value) return f.active(t);
  else return true;
}

// generic tile kernel: transforms b0 .. b0 + tb - 1 of `batch`, loader ld(b, j), storer st(b, k, v)
template <class LD, class ST>
__global__ void __launch_bounds__(1024) fft_tile_kernel(FftDesc d, int tb, int batch, int sign, int load_jfast,
                                                        int store_jfast, LD ld, ST st) {
  using C = ElemOf<LD>;
  extern __shared__ __align__(16) unsigned char fft_sm_raw[];
  C* sm = reinterpret_cast<C*>(fft_sm_raw);
  pdl_enter();
  const int b0 = blockIdx.x * tb;
  const int ntr = min(tb, batch - b0);
  if constexpr (HasActive<LD>::value || HasActive<ST>::value) {
    bool any = false;
    for (int t = 0; t < ntr && !any; ++t) any = active_of(ld, b0 + t) && active_of(st, b0 + t);
    if (!any) return;  // block-uniform
  }
  const int L = d.L, n = tb * L;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    int t, j;
    if (load_jfast) { j = idx % L; t = idx / L; } else { t = idx % tb; j = idx / tb; }
    sm[j * tb + t] = (t < ntr) ? ld(b0 + t, (int64_t)j) : czero<C>();
  }
  __syncthreads();
  fft_smem(sm, d, tb, sign);
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    int t, j;
    if (store_jfast) { j = idx % L; t = idx / L; } else { t = idx % tb; j = idx / tb; }
    if (t < ntr) st(b0 + t, (int64_t)j, sm[j * tb + t]);
  }
}

// four-step adapters ---------------------------------------------------------------------------
template <class LD>
struct ColLoad {  // transform bb = b * L2 + j2, element j1 -> user element j1 * L2 + j2 of transform b
  LD ld;
  int64_t L2;
  __device__ ElemOf<LD> operator()(int bb, int64_t j1) const {
    int64_t b = bb / L2, j2 = bb % L2;
    return ld((int)b, j1 * L2 + j2);
  }
  template <class X = LD, class = std::enable_if_t<HasActive<X>::value>>
  __device__ bool active(int bb) const { return ld.active((int)(bb / L2)); }
};
template <class C>
struct ColStore {  // tmp[b * L + k1 * L2 + j2] = v * w_L^{sign j2 k1}
  C* tmp;
  const C* twL;
  int64_t L, L2;
  int sign;
  __device__ void operator()(int bb, int64_t k1, C v) const {
    int64_t b = bb / L2, j2 = bb % L2;
    int64_t e = (j2 * k1) % L;
    C w = tw_at(twL, e);
    if (sign < 0) w.y = -w.y;
    tmp[b * L + k1 * L2 + j2] = cmul(v, w);
  }
};
template <class C>
struct RowLoad {  // transform bb = b * L1 + k1, element j2 -> tmp[b * L + k1 * L2 + j2]
  const C* tmp;
  int64_t L, L1, L2;
  __device__ C operator()(int bb, int64_t j2) const {
    int64_t b = bb / L1, k1 = bb % L1;
    return tmp[b * L + k1 * L2 + j2];
  }
};
template <class ST>
struct RowStore {  // output k = k1 + L1 * k2 of transform b
  ST st;
  int64_t L1;
  template <class C>
  __device__ void operator()(int bb, int64_t k2, C v) const {
    int64_t b = bb / L1, k1 = bb % L1;
    st((int)b, k1 + L1 * k2, v);
  }
  template <class X = ST, class = std::enable_if_t<HasActive<X>::value>>
  __device__ bool active(int bb) const { return st.active((int)(bb / L1)); }
};

// host helpers ----------------------------------------------------------------------------------
inline void fft_tile_geometry(int L, int want_tb, int& tb, int& threads) {
  tb = std::max(1, want_tb);
  while (tb > 1 && tb * L > 8192) tb >>= 1;
  int need = (tb * L + 7) / 8;
  threads = std::max(32, ((need + 31) / 32) * 32);
  threads = std::min(threads, 1024);
}

template <class LD, class ST>
inline cudaError_t launch_tile(const FftDesc& d, int want_tb, int batch, int sign, int ljf, int sjf, LD ld, ST st,
                               cudaStream_t s) {
  using C = ElemOf<LD>;
  if (batch <= 0) return cudaSuccess;
  int tb, threads;
  fft_tile_geometry(d.L, want_tb, tb, threads);
  size_t smem = sizeof(C) * (size_t)tb * d.L;
  // the dynamic shared-memory limit is a per-device function attribute: set it once per device (bit
  // dev of a mask kept per template instantiation; devices beyond 63 set it on every launch)
  static std::atomic<unsigned long long> attr_set{0ULL};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  const unsigned long long bit = dev < 64 ? (1ULL << dev) : 0ULL;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    cudaError_t e = cudaFuncSetAttribute(fft_tile_kernel<LD, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         8192 * (int)sizeof(C));
    if (e != cudaSuccess) return e;
    attr_set.fetch_or(bit, std::memory_order_acq_rel);
  }
  int blocks = (batch + tb - 1) / tb;
  cudaError_t e = launch_k(pdl_enabled(), fft_tile_kernel<LD, ST>, dim3(blocks), dim3(threads), smem, s, d, tb, batch,
                           sign, ljf, sjf, ld, st);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Run `batch` transforms of plan p in the precision of the loader's element type.  tmp must hold batch * L
// values of that type when p.four.  Returns the number of kernels launched (negative on a launch error).
template <class LD, class ST>
inline int fft_run(const FftPlan& p, int batch, int sign, LD ld, ST st, ElemOf<LD>* tmp, cudaStream_t s) {
  using C = ElemOf<LD>;
  if (!p.four) {
    int want = p.L >= p.tile ? 1 : (int)(p.tile / p.L);
    return launch_tile(p.d1, want, batch, sign, /*ljf*/ 1, /*sjf*/ 1, ld, st, s) == cudaSuccess ? 1 : -1;
  }
  ColLoad<LD> cl{ld, p.L2};
  ColStore<C> cs{tmp, Tw<C>::inter(p), p.L, p.L2, sign};
  if (launch_tile(p.d1, 8, (int)(batch * p.L2), sign, 0, 0, cl, cs, s) != cudaSuccess) return -1;
  RowLoad<C> rl{tmp, p.L, p.L1, p.L2};
  RowStore<ST> rs{st, p.L1};
  if (launch_tile(p.d2, 8, (int)(batch * p.L1), sign, 1, 0, rl, rs, s) != cudaSuccess) return -1;
  return 2;
}

// radix schedule for a 7-smooth length (8s first unless radix_max is 4, then 4 / 2, then 7s, 5s and 3s)
inline bool fft_factor(int L, FftDesc& d, int radix_max = 8) {
  d.L = L;
  d.nst = 0;
  int v = L;
  while (radix_max >= 8 && v % 8 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 8; v /= 8; }
  while (v % 4 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 4; v /= 4; }
  while (v % 2 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 2; v /= 2; }
  while (v % 7 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 7; v /= 7; }
  while (v % 5 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 5; v /= 5; }
  while (v % 3 == 0 && d.nst < FFT_MAX_STAGES) { d.rad[d.nst++] = 3; v /= 3; }
  return v == 1;
}

// split L = L1 * L2 with both factors <= FFT_TILE_MAX, as balanced as the factors allow
inline bool fft_split(int64_t L, int64_t& L1, int64_t& L2) {
  std::vector<int> f;
  int64_t v = L;
  for (int q : {2, 3, 5, 7})
    while (v % q == 0) { f.push_back(q); v /= q; }
  if (v != 1) return false;
  // greedy: put the largest factors alternately; then fix the balance
  L1 = 1;
  L2 = 1;
  std::sort(f.rbegin(), f.rend());
  for (int q : f) {
    if (L1 <= L2) L1 *= q; else L2 *= q;
  }
  return L1 <= FFT_TILE_MAX && L2 <= FFT_TILE_MAX;
}

}  // namespace tikh
