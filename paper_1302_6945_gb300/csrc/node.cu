// node.cu -- internal nodes of Algorithm 1 with paired interleaving (Sec. 4.3, 5.1).
//
// A node (a, s, L) splits into the left child (a, 2s, L/2) and the right child (a+s, 2s, L/2).
// Step 2: the left basis B_L is evaluated at the right child's nodes omega^{beta + 2s j}, j < L/2,
// beta in {a+s, a+s+1}: twist by omega^{beta t}, fold modulo L/2, DFT of length L/2 (the
// cancellation of roots of unity that Sec. 4.3 and Fig. 5 rely on); then every right condition
// phi <- phi B_L(sigma).
// Step 4: B = B_L B_R by length-P DFTs, P > the largest entry degree allowed by the tau-degrees,
// trimmed to entry (i,j) degree bounds and carried with power-of-two column scales.
#include "internal.h"

namespace tikh {

__device__ __forceinline__ int entry_bound_dev(const int* din, const int* dout, int i, int j) {
  int amax = 0;
  bool have = false;
  for (int c = 0; c < 5; ++c)
    if (dout[c] > din[c]) { amax = have ? max(amax, dout[c]) : dout[c]; have = true; }
  if (dout[j] > din[j]) return dout[j] - din[i];
  int acc = have ? amax - din[i] : -1;
  if (i == j && acc < 0) acc = 0;
  return min(acc, dout[j] - din[i]);
}

// ------------------------------------------------------------------------------------------------
// step 2
// ------------------------------------------------------------------------------------------------
struct LoadTwistFold {  // batch b = 2E + c
  BasisBuf B;
  const cd* wN;
  int64_t N, Lr, beta0;
  __device__ cd operator()(int b, int64_t u) const {
    int E = b >> 1, c = b & 1;
    int64_t beta = beta0 + c;
    int64_t len = B.len[E];
    cd acc = mkc(0.0, 0.0);
    for (int64_t t = u; t < len; t += Lr) acc = cfma(B.c[E * B.cap + t], tw_at(wN, (beta * t) % N), acc);
    return cscale(acc, col_scale_from_bits(B.colmax[E % 5]));
  }
};
struct StoreEval {
  cd* out;
  int64_t Lr;
  __device__ void operator()(int b, int64_t j, cd v) const { out[(int64_t)b * Lr + j] = v; }
};

// phi <- phi B_L(sigma) for both conditions of every right-child node
__global__ void k_eval_update(cd* R, const cd* __restrict__ vals, int64_t a0, int64_t s2, int64_t Lr) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 2 * Lr; g += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(g % 2);
    int64_t j = g / 2;
    int64_t e = a0 + c + s2 * j;
    cd V[25];
#pragma unroll
    for (int E = 0; E < 25; ++E) V[E] = vals[((int64_t)E * 2 + c) * Lr + j];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      cd* r = R + e * 10 + f * 5;
      cd in[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) in[i] = r[i];
#pragma unroll
      for (int col = 0; col < 5; ++col) {
        cd acc = mkc(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 5; ++i) acc = cfma(in[i], V[i * 5 + col], acc);
        r[col] = acc;
      }
    }
  }
}

int launch_eval(Plan& P, const Step& st) {
  const FftPlan& F = P.ffts[st.fft];
  const int64_t Lr = st.L / 2;
  const BasisBuf& BL = P.buf[st.depth + 1][0];
  int r = fft_run(F, 50, +1, LoadTwistFold{BL, P.wN, P.N, Lr, st.a + st.s}, StoreEval{P.evalv, Lr}, P.etmp, P.stream);
  if (r < 0) return TIKH_ECUDA;
  int blocks = (int)std::min<int64_t>((2 * Lr + 127) / 128, 4096);
  k_eval_update<<<blocks, 128, 0, P.stream>>>(P.R, P.evalv, st.a + st.s, 2 * st.s, Lr);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return r + 1;
}

// ------------------------------------------------------------------------------------------------
// step 4
// ------------------------------------------------------------------------------------------------
struct LoadPad {  // batch b < 25: B_L entry b; b >= 25: B_R entry b - 25; zero-padded to P
  BasisBuf BL, BR, OUT;
  const int* dstack_d;  // delta_in of the node
  const int* delta;     // delta_out
  int* status;
  int64_t P;
  __device__ cd operator()(int b, int64_t t) const {
    if (b == 0 && t == 0) {
      // guard: the transform length must exceed every entry degree of the product
      int D = -1;
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) D = max(D, entry_bound_dev(dstack_d, delta, i, j));
      for (int E = 0; E < 25; ++E) D = max(D, max(BL.len[E], BR.len[E]) - 1);
      if (D >= P) set_status(status, ST_DEGREE);
      for (int j = 0; j < 5; ++j) OUT.colmax[j] = 0ULL;
    }
    const BasisBuf& B = b < 25 ? BL : BR;
    int E = b < 25 ? b : b - 25;
    if (t >= B.len[E]) return mkc(0.0, 0.0);
    return cscale(B.c[E * B.cap + t], col_scale_from_bits(B.colmax[E % 5]));
  }
};
struct StoreSpec {
  cd* FA;
  cd* FB;
  int64_t P;
  __device__ void operator()(int b, int64_t k, cd v) const {
    if (b < 25) FA[(int64_t)b * P + k] = v;
    else FB[(int64_t)(b - 25) * P + k] = v;
  }
};
struct StorePlain2 {
  cd* out;
  int64_t P;
  __device__ void operator()(int b, int64_t k, cd v) const { out[(int64_t)b * P + k] = v; }
};
struct LoadProduct {  // output entry b = 5i + j: sum_t FA[5i+t] FB[5t+j]
  const cd* FA;
  const cd* FB;
  int64_t P;
  __device__ cd operator()(int b, int64_t u) const {
    int i = b / 5, j = b % 5;
    cd acc = mkc(0.0, 0.0);
#pragma unroll
    for (int t = 0; t < 5; ++t) acc = cfma(FA[(int64_t)(5 * i + t) * P + u], FB[(int64_t)(5 * t + j) * P + u], acc);
    return acc;
  }
};

// trim to the degree bounds, scale by 1/P, record column maxima and lengths
__global__ void k_prod_finish(const cd* __restrict__ FC, int64_t P, BasisBuf OUT, const int* dstack_d,
                              const int* delta, int* status) {
  const int E = blockIdx.y, i = E / 5, j = E % 5;
  __shared__ int want_s;
  __shared__ double red[32];
  if (threadIdx.x == 0) {
    int bnd = entry_bound_dev(dstack_d, delta, i, j);
    int64_t want = bnd < 0 ? 0 : (int64_t)bnd + 1;
    if (want > P) want = P;
    if (want > OUT.cap) { set_status(status, ST_DEGREE); want = OUT.cap; }
    want_s = (int)want;
    if (blockIdx.x == 0) OUT.len[E] = (int)want;
  }
  __syncthreads();
  const int64_t want = want_s;
  const double inv = 1.0 / (double)P;
  double mx = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < want; t += (int64_t)gridDim.x * blockDim.x) {
    cd v = cscale(FC[(int64_t)E * P + t], inv);
    OUT.c[(int64_t)E * OUT.cap + t] = v;
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    if (mx > 0.0) atomicMax(OUT.colmax + j, (unsigned long long)__double_as_longlong(mx));
  }
}

int launch_prod(Plan& P, const Step& st) {
  const FftPlan& F = P.ffts[st.fft];
  const BasisBuf& BL = P.buf[st.depth + 1][0];
  const BasisBuf& BR = P.buf[st.depth + 1][1];
  const BasisBuf& OUT = P.buf[st.depth][st.side];
  const int* dsd = P.dstack + st.depth * 5;
  int nl = 0, r;
  LoadPad lp{BL, BR, OUT, dsd, P.delta, P.status, st.P};
  if ((r = fft_run(F, 50, +1, lp, StoreSpec{P.FA, P.FB, st.P}, P.ptmp, P.stream)) < 0) return TIKH_ECUDA;
  nl += r;
  if ((r = fft_run(F, 25, -1, LoadProduct{P.FA, P.FB, st.P}, StorePlain2{P.FC, st.P}, P.ptmp, P.stream)) < 0)
    return TIKH_ECUDA;
  nl += r;
  int bx = (int)std::min<int64_t>((st.P + 255) / 256, 64);
  k_prod_finish<<<dim3(bx, 25), 256, 0, P.stream>>>(P.FC, st.P, OUT, dsd, P.delta, P.status);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return nl + 1;
}

}  // namespace tikh
