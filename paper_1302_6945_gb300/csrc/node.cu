// node.cu -- internal nodes of Algorithm 1 with paired interleaving (Sec. 4.3, 6.1).
//
// A node (a, s, L) splits into the left child (a, 2s, L/2) and the right child (a+s, 2s, L/2).
// Step 2: the left basis B_L is evaluated at the right child's nodes omega^{beta + 2s j}, j < L/2,
// beta in {a+s, a+s+1}: twist by omega^{beta t}, fold modulo L/2, DFT of length L/2 (the
// cancellation of roots of unity that Sec. 4.3 and Sec. 6.1 rely on); then every right condition
// phi <- phi B_L(sigma).
// Step 4: B = B_L B_R by length-P DFTs, P > the largest entry degree allowed by the tau-degrees,
// trimmed to entry (i,j) degree bounds and carried with power-of-two column scales.
// In the FP32 precision pattern the FFT forms of both steps run in FP32 (complex64 spectra, FP32
// pointwise products and updates); the direct small-node forms, the leaves and the basis stay FP64.
// All problems of a batch are processed by the same launches: transform index = problem * 2 W^2 (or W^2)
// + entry, grid.y / grid.z = problem for the element-wise kernels.  W = 5 (the l2 and Toeplitz-Gramian
// problems, two condition sets per node) or 7 (the general problem, three sets per node).
#include "internal.h"

namespace tikh {

template <int W>
__device__ __forceinline__ int entry_bound_dev(const int* din, const int* dout, int i, int j) {
  int amax = 0;
  bool have = false;
  for (int c = 0; c < W; ++c)
    if (dout[c] > din[c]) { amax = have ? max(amax, dout[c]) : dout[c]; have = true; }
  if (dout[j] > din[j]) return dout[j] - din[i];
  int acc = have ? amax - din[i] : -1;
  if (i == j && acc < 0) acc = 0;
  return min(acc, dout[j] - din[i]);
}

// ------------------------------------------------------------------------------------------------
// step 2
// ------------------------------------------------------------------------------------------------
// The FFT path of steps 2 and 4 runs in the plan's stage precision C: complex128 (cd), or complex64 (cf)
// in the FP32 precision pattern (FP32 arithmetic and accumulation; the basis stays FP64 and so do the
// residual rows, which the FP64 leaves read).
template <class C>
__device__ __forceinline__ C twiddle_of(const cd* wN, const cf* wN32, int64_t i);
template <>
__device__ __forceinline__ cd twiddle_of<cd>(const cd* wN, const cf*, int64_t i) { return tw_at(wN, i); }
template <>
__device__ __forceinline__ cf twiddle_of<cf>(const cd*, const cf* wN32, int64_t i) { return tw_at(wN32, i); }

// columns pivoted between two degree vectors (bit j: dout_j > din_j); a single-point factor of Eq. (spbasis)
// changes only its pivot column and leaves every other row of the basis an identity row, so the rows of a
// node's basis outside the columns pivoted in that node are exactly identity rows (scaled by the lazy
// column scales)
template <int W>
__device__ __forceinline__ unsigned pivoted_cols(const int* din, const int* dout) {
  unsigned m = 0u;
#pragma unroll
  for (int j = 0; j < W; ++j) m |= (dout[j] > din[j] ? 1u : 0u) << j;
  return m;
}

// Step 2 at a node of depth `depth`: the rows of B_L outside the columns pivoted in the left child (from
// delta_in of the node, dstack[depth], to the current delta) are identity rows, whose evaluation is the
// constant diagonal; their transforms are skipped
template <int W>
struct EvalNeed {
  const int* dstack;
  const int* delta;
  int depth;
  __device__ unsigned sl(int pb) const {
    return pivoted_cols<W>(dstack + (pb * MAX_DEPTH + depth) * DSTR, delta + DSTR * pb);
  }
  __device__ bool active(int t) const {  // transform t = 2 W^2 pb + 2E + c, E = W i + j
    const int pb = t / (2 * W * W), i = ((t % (2 * W * W)) >> 1) / W;
    return (sl(pb) >> i) & 1u;
  }
};

template <class C, int W>
struct LoadTwistFold {  // transform t = 2 W^2 pb + 2E + c
  BasisBuf B;
  BasisBuf OUT;  // this node's output slot: its column maxima are reset here, before the product
  const cd* wN;
  const cf* wN32;
  int64_t N, Lr, beta0;
  EvalNeed<W> need;
  __device__ bool active(int t) const { return need.active(t); }
  __device__ C operator()(int t, int64_t u) const {
    int pb = t / (2 * W * W), b = t % (2 * W * W);
    if (b == 0 && u == 0)
      for (int j = 0; j < W; ++j) OUT.mp(pb)[j] = 0ULL;
    int E = b >> 1, c = b & 1;
    int64_t beta = beta0 + c;
    int64_t len = B.lp(pb)[E];
    const cd* src = B.cp(pb) + E * B.cap;
    C acc = czero<C>();
    // twiddle index (beta q) mod N advanced by (beta Lr) mod N per fold term (one 64-bit modulo each)
    int64_t ix = (beta * u) % N;
    const int64_t stepx = (beta * Lr) % N;
    for (int64_t q = u; q < len; q += Lr) {
      acc = cfma(cfrom<C>(src[q]), twiddle_of<C>(wN, wN32, ix), acc);
      ix += stepx;
      if (ix >= N) ix -= N;
    }
    return cscale(acc, (decltype(acc.x))col_scale_from_bits(B.mp(pb)[E % W]));
  }
};
template <class C, int W>
struct StoreEval {
  C* out;
  int64_t Lr;
  EvalNeed<W> need;
  __device__ bool active(int t) const { return need.active(t); }
  __device__ void operator()(int t, int64_t j, C v) const { out[(int64_t)t * Lr + j] = v; }
};

// phi <- phi B_L(sigma) for the NS conditions of every right-child node (in C's precision; the rows are
// stored back in FP64).  An identity row i of B_L (skipped by the transforms) evaluates to its constant
// diagonal, computed here as the twist-fold transform computes it.  Also resets this node's column maxima
// (the product accumulates them).
template <class C, int W, int NS>
__global__ void k_eval_update(cd* R, const C* __restrict__ vals, int64_t N, int64_t a0, int64_t s2, int64_t Lr,
                              BasisBuf BL, BasisBuf OUT, EvalNeed<W> need) {
  pdl_enter();
  const int pb = blockIdx.y;
  if (blockIdx.x == 0 && threadIdx.x < W) OUT.mp(pb)[threadIdx.x] = 0ULL;
  const unsigned SL = need.sl(pb);
  C D[W];  // the constant evaluation of each identity row's diagonal
#pragma unroll
  for (int i = 0; i < W; ++i) {
    D[i] = czero<C>();
    if (!((SL >> i) & 1u) && BL.lp(pb)[i * W + i] >= 1)
      D[i] = cscale(cfrom<C>(BL.cp(pb)[(int64_t)(i * W + i) * BL.cap]),
                    (decltype(D[i].x))col_scale_from_bits(BL.mp(pb)[i]));
  }
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 2 * Lr; g += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(g % 2);
    int64_t j = g / 2;
    int64_t e = a0 + c + s2 * j;
    C V[W * W];
#pragma unroll
    for (int E = 0; E < W * W; ++E) {
      const int i = E / W;
      V[E] = ((SL >> i) & 1u) ? vals[((int64_t)pb * (2 * W * W) + E * 2 + c) * Lr + j]
                              : (E % W == i ? D[i] : czero<C>());
    }
#pragma unroll
    for (int f = 0; f < NS; ++f) {
      cd* r = R + ((int64_t)pb * N + e) * (NS * W) + f * W;
      C in[W];
#pragma unroll
      for (int i = 0; i < W; ++i) in[i] = cfrom<C>(r[i]);
#pragma unroll
      for (int col = 0; col < W; ++col) {
        C acc = czero<C>();
#pragma unroll
        for (int i = 0; i < W; ++i) acc = cfma(in[i], V[i * W + col], acc);
        r[col] = mkc((double)acc.x, (double)acc.y);
      }
    }
  }
}

// Small nodes: B_L evaluated at each right-child node, then the residual update of that node's NS
// conditions, in one launch.  Block = one node (g = 2j + c), W^2 entries x G lanes: lane gl evaluates
// the coefficient chunk [gl C, gl C + C) of its entry by Horner, multiplies by z^(gl C) (twiddle
// table) and the G lanes are added by shuffles; then NS W threads form phi <- phi B_L(sigma).
template <int G, int W, int NS>
__global__ void __launch_bounds__(W * W * G) k_eval_direct(BasisBuf BL, BasisBuf OUT, cd* R, const cd* __restrict__ wN,
                                                           int64_t N, int64_t a0, int64_t s2) {
  __shared__ cd V[W * W];
  __shared__ cd Rs[NS * W];
  pdl_enter();
  const int pb = blockIdx.y, tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t e = a0 + (g & 1) + s2 * (g >> 1);
  if (g == 0 && tid < W) OUT.mp(pb)[tid] = 0ULL;  // the parent's column maxima, rebuilt by its product
  if (tid < NS * W) Rs[tid] = R[((int64_t)pb * N + e) * (NS * W) + tid];
  const int E = tid / G, gl = tid - E * G;
  const int len = BL.lp(pb)[E];
  const int C = (len + G - 1) / G;
  const int cnt = min(C, len - gl * C);
  const cd z = wN[e];
  const cd* c = BL.cp(pb) + (int64_t)E * BL.cap + (int64_t)gl * C;
  cd v = mkc(0.0, 0.0);
  for (int t = cnt - 1; t >= 0; --t) v = cfma(v, z, c[t]);
  if (G > 1) {
    if (gl > 0 && cnt > 0) v = cmul(v, tw_at(wN, (e * (int64_t)(gl * C)) % N));
    const int wbase = tid & ~31;
    const int nw = min(32, (int)blockDim.x - wbase);
    const unsigned mask = nw == 32 ? 0xffffffffu : ((1u << nw) - 1u);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(mask, v.x, o);
      v.y += __shfl_xor_sync(mask, v.y, o);
    }
  }
  if (gl == 0) V[E] = cscale(v, col_scale_from_bits(BL.mp(pb)[E % W]));
  __syncthreads();
  if (tid < NS * W) {  // (condition f, column): phi <- phi B_L(sigma)
    const int f = tid / W, col = tid % W;
    cd acc = mkc(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < W; ++i) acc = cfma(Rs[f * W + i], V[i * W + col], acc);
    R[((int64_t)pb * N + e) * (NS * W) + f * W + col] = acc;
  }
}

template <int W, int NS>
static int launch_eval_t(Plan& P, const Step& st) {
  const int64_t Lr = st.L / 2;
  const BasisBuf& BL = P.buf[st.depth + 1][0];
  const BasisBuf& OUT = P.buf[st.depth][st.side];
  constexpr int WW = W * W;
  if (Lr <= P.eval_direct_max) {
    const dim3 grid((unsigned)(2 * Lr), (unsigned)P.nb);
    const int64_t cap = BL.cap, a0 = st.a + st.s, s2 = 2 * st.s;
    cudaStream_t s = P.stream;
    const bool pdl = pdl_enabled();
    if (cap <= 8) launch_k(pdl, k_eval_direct<1, W, NS>, grid, dim3(WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    else if (cap <= 24) launch_k(pdl, k_eval_direct<2, W, NS>, grid, dim3(2 * WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    else if (cap <= 48) launch_k(pdl, k_eval_direct<4, W, NS>, grid, dim3(4 * WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    else if (cap <= 96) launch_k(pdl, k_eval_direct<8, W, NS>, grid, dim3(8 * WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    else if (cap <= 192 || W > 5)  // 16 lanes per entry at most for the 7 x 7 basis (784 threads)
      launch_k(pdl, k_eval_direct<16, W, NS>, grid, dim3(16 * WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    else launch_k(pdl, k_eval_direct<32, W, NS>, grid, dim3(32 * WW), 0, s, BL, OUT, P.R, P.wN, P.N, a0, s2);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  const FftPlan& F = P.ffts[st.fft];
  dim3 grid((unsigned)std::min<int64_t>((2 * Lr + 127) / 128, 4096), (unsigned)P.nb);
  const EvalNeed<W> need{P.dstack, P.delta, st.depth};
  int r;
  if constexpr (W == 5) {
    if (P.stage32) {
      cf* ev = reinterpret_cast<cf*>(P.evalv);
      r = fft_run(F, 2 * WW * P.nb, +1, LoadTwistFold<cf, W>{BL, OUT, P.wN, P.wN32, P.N, Lr, st.a + st.s, need},
                  StoreEval<cf, W>{ev, Lr, need}, reinterpret_cast<cf*>(P.etmp), P.stream);
      if (r < 0) return TIKH_ECUDA;
      launch_k(pdl_enabled(), k_eval_update<cf, W, NS>, grid, dim3(128), 0, P.stream, P.R, (const cf*)ev, P.N,
               st.a + st.s, 2 * st.s, Lr, BL, OUT, need);
      if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
      return r + 1;
    }
  }
  r = fft_run(F, 2 * WW * P.nb, +1, LoadTwistFold<cd, W>{BL, OUT, P.wN, P.wN32, P.N, Lr, st.a + st.s, need},
              StoreEval<cd, W>{P.evalv, Lr, need}, P.etmp, P.stream);
  if (r < 0) return TIKH_ECUDA;
  launch_k(pdl_enabled(), k_eval_update<cd, W, NS>, grid, dim3(128), 0, P.stream, P.R, (const cd*)P.evalv, P.N,
           st.a + st.s, 2 * st.s, Lr, BL, OUT, need);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return r + 1;
}

int launch_eval(Plan& P, const Step& st) { return P.w == 7 ? launch_eval_t<7, 3>(P, st) : launch_eval_t<5, 2>(P, st); }

// ------------------------------------------------------------------------------------------------
// step 4
// ------------------------------------------------------------------------------------------------
// length bound of entry (i, j) of B_L B_R from the operands' lengths: max_u len(a_iu) + len(b_uj) - 1 (the
// tau-degree bound can be far looser when the extension k is large)
template <int W>
__device__ __forceinline__ int prod_len_bound(const BasisBuf& BL, const BasisBuf& BR, int pb, int i, int j) {
  int L = 0;
  for (int u = 0; u < W; ++u) {
    const int la = BL.lp(pb)[i * W + u], lb = BR.lp(pb)[u * W + j];
    if (la > 0 && lb > 0) L = max(L, la + lb - 1);
  }
  return L;
}

// entry (i, i) of an identity row i of basis B, as its evaluations and transforms see it (column scale
// applied): the stored constant coefficient
template <int W>
__device__ __forceinline__ cd identity_diag(const BasisBuf& B, int pb, int i) {
  const int E = i * W + i;
  if (B.lp(pb)[E] < 1) return mkc(0.0, 0.0);
  return col_scaled(B.cp(pb)[(int64_t)E * B.cap], B.mp(pb)[i]);
}

// What a product B = B_L B_R at recursion depth `depth` computes.
// (1) Identity rows: rows of B_L outside the columns pivoted in the left child (S_L), and of B_R outside
// S_R, are identity rows; their transforms are skipped and the products use their constant diagonal; the
// output rows outside S_L u S_R are identity rows written directly.  S_L and S_R come from the degree
// vectors: delta_in of the node (dstack[depth]), of its right child (dstack[depth + 1]) and delta_out.
// (2) The extraction (Sec. 5) reads entries (0, j*) and (W-1, j*) of the root's basis only, j* its column
// of tau-degree 0.  When no condition of the problem was deferred, the root's product is needed for those
// two entries (rows 0 and W-1 of B_L, column j* of B_R), and the product of every other node on the right
// spine (the root's right child, its right child, ...), whose basis only enters its parent's product as
// B_R, for its column j* (all of its B_L, column j* of its B_R).  These products come after the last leaf,
// so the deferral count and the degree pattern are final when they run (mode 1: a right-spine node, 2: the
// root, 0: any other node; ndiff == nullptr: no such reduction).  With deferred conditions, or without
// the final degree pattern, every entry is computed.
template <int W>
struct ProdNeed {
  const int* ndiff;
  const int* delta;
  const int* dstack;
  int depth;
  int mode;
  __device__ int jstar(int pb) const {
    if (!ndiff || mode == 0 || ndiff[4 * pb] != 0) return -1;
    const int* d = delta + DSTR * pb;
    int js = -1, nz = 0, no = 0;
    for (int j = 0; j < W; ++j) {
      if (d[j] == 0) { js = j; ++nz; } else if (d[j] == 1) ++no;
    }
    return nz == 1 && no == W - 1 ? js : -1;
  }
  __device__ unsigned sl(int pb) const {
    return pivoted_cols<W>(dstack + (pb * MAX_DEPTH + depth) * DSTR, dstack + (pb * MAX_DEPTH + depth + 1) * DSTR);
  }
  __device__ unsigned sr(int pb) const {
    return pivoted_cols<W>(dstack + (pb * MAX_DEPTH + depth + 1) * DSTR, delta + DSTR * pb);
  }
  // operand transform t = 2 W^2 pb + b (b < W^2: B_L entry b, else B_R entry b - W^2)
  __device__ bool operand(int t) const {
    const int pb = t / (2 * W * W), b = t % (2 * W * W);
    const int js = jstar(pb);
    if (b < W * W) {
      const int i = b / W;
      return ((sl(pb) >> i) & 1u) && (js < 0 || mode == 1 || i == 0 || i == W - 1);
    }
    const int u = (b - W * W) / W, j = (b - W * W) % W;
    return ((sr(pb) >> u) & 1u) && (js < 0 || j == js);
  }
  // output entry t = W^2 pb + E: 0 nothing reads it, 1 an identity row (written directly), 2 computed
  __device__ int output(int t) const {
    const int pb = t / (W * W), e = t % (W * W), i = e / W, j = e % W;
    const int js = jstar(pb);
    if (js >= 0 && !(j == js && (mode == 1 || i == 0 || i == W - 1))) return 0;
    return (((sl(pb) | sr(pb)) >> i) & 1u) ? 2 : 1;
  }
};

template <class C, int W>
struct LoadPad {  // transform t = 2 W^2 pb + b; b < W^2: B_L entry b; else B_R entry b - W^2; zero-padded to P
  BasisBuf BL, BR;
  int64_t P;
  ProdNeed<W> need;
  __device__ C operator()(int t, int64_t q) const {
    constexpr int WW = W * W;
    int pb = t / (2 * WW), b = t % (2 * WW);
    const BasisBuf& B = b < WW ? BL : BR;
    int E = b < WW ? b : b - WW;
    if (q >= B.lp(pb)[E]) return czero<C>();
    return cfrom<C>(col_scaled(B.cp(pb)[E * B.cap + q], B.mp(pb)[E % W]));
  }
  __device__ bool active(int t) const { return need.operand(t); }
};
template <class C, int W>
struct StoreSpec {
  C* FA;
  C* FB;
  int64_t P;
  ProdNeed<W> need;
  __device__ void operator()(int t, int64_t k, C v) const {
    constexpr int WW = W * W;
    int pb = t / (2 * WW), b = t % (2 * WW);
    if (b < WW) FA[((int64_t)pb * WW + b) * P + k] = v;
    else FB[((int64_t)pb * WW + b - WW) * P + k] = v;
  }
  __device__ bool active(int t) const { return need.operand(t); }
};
template <class C, int W>
struct StorePlain2 {
  C* out;
  int64_t P;
  ProdNeed<W> need;
  __device__ void operator()(int t, int64_t k, C v) const { out[(int64_t)t * P + k] = v; }
  __device__ bool active(int t) const { return need.output(t) == 2; }
};
template <class C, int W>
struct LoadProduct {  // transform t = W^2 pb + W i + j: sum_u FA[W i + u] FB[W u + j]
  const C* FA;
  const C* FB;
  int64_t P;
  BasisBuf BL, BR;
  ProdNeed<W> need;
  __device__ bool active(int t) const { return need.output(t) == 2; }
  __device__ C operator()(int t, int64_t q) const {
    constexpr int WW = W * W;
    int pb = t / WW, e = t % WW, i = e / W, j = e % W;
    const C* a = FA + (int64_t)pb * WW * P;
    const C* b = FB + (int64_t)pb * WW * P;
    // an identity row's transform is its constant diagonal at every bin (the transform of a constant)
    const unsigned SL = need.sl(pb), SR = need.sr(pb);
    const bool li = (SL >> i) & 1u;
    const C dl = li ? czero<C>() : cfrom<C>(identity_diag<W>(BL, pb, i));
    C acc = czero<C>();
#pragma unroll
    for (int u = 0; u < W; ++u) {
      const C x = li ? a[(int64_t)(W * i + u) * P + q] : (u == i ? dl : czero<C>());
      const C y = ((SR >> u) & 1u) ? b[(int64_t)(W * u + j) * P + q]
                                  : (u == j ? cfrom<C>(identity_diag<W>(BR, pb, u)) : czero<C>());
      acc = cfma(x, y, acc);
    }
    return acc;
  }
};

// max(|Re|, |Im|) as the bit pattern of a non-negative double, by integer operations (no FP64 instruction:
// non-negative doubles order like their bit patterns)
__device__ __forceinline__ unsigned long long absmax_bits(cd v) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffULL;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffULL;
  return a > b ? a : b;
}

// trim to the degree bounds, scale by 1/P (in FP64), record column maxima and lengths; identity rows
// written directly; the guard that the transform length exceeds every entry degree of the product
template <class C, int W>
__global__ void k_prod_finish(const C* __restrict__ FC, int64_t P, BasisBuf BL, BasisBuf BR, BasisBuf OUT,
                              const int* dstack, int depth, const int* delta, int* status, ProdNeed<W> need) {
  const int E = blockIdx.y, i = E / W, j = E % W, pb = blockIdx.z;
  __shared__ int want_s;
  __shared__ unsigned long long red[32];
  pdl_enter();
  if (blockIdx.x == 0 && E == 0 && threadIdx.x == 0) {  // no wrap-around (else a re-plan with more slack)
    const int* din = dstack + (pb * MAX_DEPTH + depth) * DSTR;
    const int* dout = delta + DSTR * pb;
    int D = -1;
    for (int a = 0; a < W; ++a)
      for (int c = 0; c < W; ++c)
        D = max(D, min(entry_bound_dev<W>(din, dout, a, c), prod_len_bound<W>(BL, BR, pb, a, c) - 1));
    for (int e = 0; e < W * W; ++e) D = max(D, max(BL.lp(pb)[e], BR.lp(pb)[e]) - 1);  // operands fit
    if (D >= P) set_status(status, ST_DEGREE);
  }
  const int code = need.output(pb * W * W + E);
  if (code != 2) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
      if (code == 1 && i == j) {  // identity row: its diagonal is the product of the operands' diagonals
        const cd v = cmul(identity_diag<W>(BL, pb, i), identity_diag<W>(BR, pb, i));
        OUT.cp(pb)[(int64_t)E * OUT.cap] = v;
        OUT.lp(pb)[E] = 1;
        const unsigned long long m = absmax_bits(v);
        if (m > 0ULL) atomicMax(OUT.mp(pb) + j, m);
      } else {
        OUT.lp(pb)[E] = 0;  // off the diagonal of an identity row, or an entry nothing reads
      }
    }
    return;
  }
  if (threadIdx.x == 0) {
    int bnd = entry_bound_dev<W>(dstack + (pb * MAX_DEPTH + depth) * DSTR, delta + DSTR * pb, i, j);
    int64_t want = bnd < 0 ? 0 : (int64_t)bnd + 1;
    want = min(want, (int64_t)prod_len_bound<W>(BL, BR, pb, i, j));
    if (want > P) want = P;
    if (want > OUT.cap) { set_status(status, ST_DEGREE); want = OUT.cap; }
    want_s = (int)want;
    if (blockIdx.x == 0) OUT.lp(pb)[E] = (int)want;
  }
  __syncthreads();
  const int64_t want = want_s;
  const double inv = 1.0 / (double)P;
  const C* src = FC + ((int64_t)pb * (W * W) + E) * P;
  cd* dst = OUT.cp(pb) + (int64_t)E * OUT.cap;
  unsigned long long mx = 0ULL;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < want; t += (int64_t)gridDim.x * blockDim.x) {
    const C w = src[t];
    cd v = mkc((double)w.x * inv, (double)w.y * inv);
    dst[t] = v;
    const unsigned long long m = absmax_bits(v);
    mx = m > mx ? m : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long q = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = q > mx ? q : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    if (mx > 0ULL) atomicMax(OUT.mp(pb) + j, mx);
  }
}

// Small nodes: schoolbook product B = B_L B_R.  Block = (output entry E = (i, j), tile of PD_TC
// coefficients, problem); warp w computes coefficient t = tile PD_TC + w, its lanes splitting the
// terms (u, q) of sum_u sum_q a_iu[q] b_uj[t - q] and a shuffle reduction adding them, so each lane's
// FP64 chain is short and the product spreads over W^2 ceil(P / PD_TC) blocks.  Row i of B_L and
// column j of B_R are staged in shared memory with their column scales applied.  Output trimmed to
// the degree bound; column maxima accumulated (reset by this node's evaluation step).
constexpr int PD_TC = 8;
template <int W>
__global__ void __launch_bounds__(32 * PD_TC) k_prod_direct(BasisBuf BL, BasisBuf BR, BasisBuf OUT, const int* dstack,
                                                             int depth, const int* delta, int* status, int ntile,
                                                             ProdNeed<W> need) {
  extern __shared__ cd pd_sh[];  // A: W x BL.cap, then B: W x BR.cap
  const int E = blockIdx.x / ntile, tile = blockIdx.x % ntile;
  const int i = E / W, j = E % W, pb = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  __shared__ int want_s, ll[W], lr[W];
  __shared__ double red[PD_TC];
  pdl_enter();
  if (need.output(pb * W * W + E) == 0) {  // an entry of the root's basis that nothing reads
    if (tid == 0 && tile == 0) OUT.lp(pb)[E] = 0;
    return;
  }
  if (tid < W) {
    ll[tid] = BL.lp(pb)[i * W + tid];
    lr[tid] = BR.lp(pb)[tid * W + j];
  }
  if (tid == 0) {
    int bnd = entry_bound_dev<W>(dstack + (pb * MAX_DEPTH + depth) * DSTR, delta + DSTR * pb, i, j);
    int want = bnd < 0 ? 0 : bnd + 1;
    want = min(want, prod_len_bound<W>(BL, BR, pb, i, j));
    if (want > OUT.cap) { set_status(status, ST_DEGREE); want = (int)OUT.cap; }
    want_s = want;
    if (tile == 0) OUT.lp(pb)[E] = want;
  }
  __syncthreads();
  const int want = want_s, t0 = tile * PD_TC;
  if (t0 >= want) return;  // block-uniform
  const int tmax = min(want, t0 + PD_TC);
  const int capL = (int)BL.cap, capR = (int)BR.cap;
  cd* As = pd_sh;
  cd* Bs = pd_sh + W * capL;
  for (int idx = tid; idx < W * capL; idx += blockDim.x) {
    const int u = idx / capL, q = idx - u * capL;
    if (q < min(ll[u], tmax))
      As[idx] = col_scaled(BL.cp(pb)[(int64_t)(i * W + u) * capL + q], BL.mp(pb)[u]);
  }
  const unsigned long long sr = BR.mp(pb)[j];
  for (int idx = tid; idx < W * capR; idx += blockDim.x) {
    const int u = idx / capR, q = idx - u * capR;
    if (q < min(lr[u], tmax)) Bs[idx] = col_scaled(BR.cp(pb)[(int64_t)(u * W + j) * capR + q], sr);
  }
  __syncthreads();
  double mx = 0.0;
  const int t = t0 + w;
  if (t < tmax) {  // warp-uniform
    int lo[W], pre[W], tot = 0;
#pragma unroll
    for (int u = 0; u < W; ++u) {
      lo[u] = max(0, t - lr[u] + 1);
      const int hi = min(t, ll[u] - 1);
      pre[u] = tot;
      tot += max(0, hi - lo[u] + 1);
    }
    cd acc = mkc(0.0, 0.0);
    for (int k = lane; k < tot; k += 32) {
      int u = 0, base = 0, l0 = lo[0];
#pragma unroll
      for (int v = 1; v < W; ++v)
        if (k >= pre[v]) { u = v; base = pre[v]; l0 = lo[v]; }
      const int q = l0 + (k - base);
      acc = cfma(As[u * capL + q], Bs[u * capR + (t - q)], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      OUT.cp(pb)[(int64_t)E * OUT.cap + t] = acc;
      mx = fmax(fabs(acc.x), fabs(acc.y));
    }
  }
  if (lane == 0) red[w] = mx;
  __syncthreads();
  if (tid == 0) {
    for (int v = 1; v < PD_TC; ++v) mx = fmax(mx, red[v]);
    if (mx > 0.0) atomicMax(OUT.mp(pb) + j, (unsigned long long)__double_as_longlong(mx));
  }
}

// the root is (a, s) = (0, 2) and a right child is (a + s, 2 s): the right spine is a = s - 2
template <int W>
static ProdNeed<W> need_of(const Plan& P, const Step& st) {
  const int mode = st.depth == 0 ? 2 : (st.a == st.s - 2 ? 1 : 0);
  return ProdNeed<W>{mode ? P.ndiff : nullptr, P.delta, P.dstack, st.depth, mode};
}

// step 4 by length-P transforms in precision C: the 2 W^2 operand spectra, W^2 pointwise products of W
// terms, W^2 inverse transforms, then the FP64 trim / scale / column maxima
template <class C, int W>
static int launch_prod_fft(Plan& P, const Step& st, const BasisBuf& BL, const BasisBuf& BR, const BasisBuf& OUT) {
  constexpr int WW = W * W;
  const FftPlan& F = P.ffts[st.fft];
  C* FA = reinterpret_cast<C*>(P.FA);
  C* FB = reinterpret_cast<C*>(P.FB);
  C* FC = reinterpret_cast<C*>(P.FC);
  C* tmp = reinterpret_cast<C*>(P.ptmp);
  int nl = 0, r;
  const ProdNeed<W> need = need_of<W>(P, st);
  LoadPad<C, W> lp{BL, BR, st.P, need};
  if ((r = fft_run(F, 2 * WW * P.nb, +1, lp, StoreSpec<C, W>{FA, FB, st.P, need}, tmp, P.stream)) < 0)
    return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(F, WW * P.nb, -1, LoadProduct<C, W>{FA, FB, st.P, BL, BR, need}, StorePlain2<C, W>{FC, st.P, need},
                   tmp, P.stream)) < 0)
    return TIKH_ECUDA;
  nl += r;
  int bx = (int)std::min<int64_t>((st.P + 255) / 256, 64);
  launch_k(pdl_enabled(), k_prod_finish<C, W>, dim3(bx, WW, P.nb), dim3(256), 0, P.stream, (const C*)FC, st.P, BL, BR,
           OUT, (const int*)P.dstack, st.depth, (const int*)P.delta, P.status, need);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return nl + 1;
}

template <int W>
static int launch_prod_t(Plan& P, const Step& st) {
  const BasisBuf& BL = P.buf[st.depth + 1][0];
  const BasisBuf& BR = P.buf[st.depth + 1][1];
  const BasisBuf& OUT = P.buf[st.depth][st.side];
  const size_t smem = sizeof(cd) * W * (size_t)(BL.cap + BR.cap);
  if (st.P <= P.prod_direct_max && smem <= 48 * 1024) {
    const int ntile = (int)((st.P + PD_TC - 1) / PD_TC);
    const ProdNeed<W> need = need_of<W>(P, st);
    launch_k(pdl_enabled(), k_prod_direct<W>, dim3(W * W * ntile, P.nb), dim3(32 * PD_TC), smem, P.stream, BL, BR,
             OUT, (const int*)P.dstack, st.depth, (const int*)P.delta, P.status, ntile, need);
    return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
  }
  if constexpr (W == 5) {
    if (P.stage32) return launch_prod_fft<cf, W>(P, st, BL, BR, OUT);
  }
  return launch_prod_fft<cd, W>(P, st, BL, BR, OUT);
}

int launch_prod(Plan& P, const Step& st) { return P.w == 7 ? launch_prod_t<7>(P, st) : launch_prod_t<5>(P, st); }

}  // namespace tikh
