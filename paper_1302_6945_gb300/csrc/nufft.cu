// nufft.cu -- the weighted Gramian of non-uniform Fourier samples (Sec. 7.4), by direct sums.
//
// K spectral samples X_k = sum_s x_s exp(-2 pi i f_k s) of a length-n signal, with density weights w_k,
// give the Tikhonov system (A^H W A + L^H L) x = A^H W X whose Gramian G_A = A^H W A is Hermitian
// Toeplitz: (G_A)_{rs} = g_{r-s} with g_d = sum_k w_k exp(+2 pi i f_k d).  Its first column g and the
// right-hand side y_s = sum_k w_k X_k exp(+2 pi i f_k s) are O(nK) sums, computed here in FP64 (one
// thread per index d = s, the samples staged through shared memory in tiles); the solve is then the
// Toeplitz-Gramian problem (tikh_solve_gramian).
#include "internal.h"

namespace tikh {

constexpr int NU_TILE = 256;

// exp(+2 pi i f d) with the phase f d reduced to [-1/2, 1/2] first (sincospi on a small argument)
__device__ __forceinline__ cd phase(double f, double d) {
  const double t = f * d;
  const double r = t - rint(t);
  double s, c;
  sincospi(2.0 * r, &s, &c);
  return mkc(c, s);
}

__global__ void __launch_bounds__(NU_TILE) k_nufft_gramian(int64_t K, const double* __restrict__ f,
                                                            const double* __restrict__ w, const cd* __restrict__ X,
                                                            int64_t n, cd* g, cd* y) {
  __shared__ double fs[NU_TILE], ws[NU_TILE];
  __shared__ cd xs[NU_TILE];
  const int64_t d = blockIdx.x * (int64_t)NU_TILE + threadIdx.x;
  cd ag = mkc(0.0, 0.0), ay = mkc(0.0, 0.0);
  for (int64_t k0 = 0; k0 < K; k0 += NU_TILE) {
    const int cnt = (int)(K - k0 < NU_TILE ? K - k0 : NU_TILE);
    __syncthreads();
    if (threadIdx.x < cnt) {
      fs[threadIdx.x] = f[k0 + threadIdx.x];
      ws[threadIdx.x] = w[k0 + threadIdx.x];
      xs[threadIdx.x] = X[k0 + threadIdx.x];
    }
    __syncthreads();
    if (d < n) {
      for (int k = 0; k < cnt; ++k) {
        const cd e = phase(fs[k], (double)d);
        ag = cfma(e, mkc(ws[k], 0.0), ag);
        ay = cfma(e, cscale(xs[k], ws[k]), ay);
      }
    }
  }
  if (d < n) {
    g[d] = ag;
    y[d] = ay;
  }
}

}  // namespace tikh

using namespace tikh;

extern "C" int tikh_nufft_gramian(int64_t K, const double* f, const double* w, const void* X, int64_t n, void* g,
                                  void* y, void* stream) {
  if (K < 1 || n < 1 || !f || !w || !X || !g || !y) return TIKH_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((n + NU_TILE - 1) / NU_TILE);
  k_nufft_gramian<<<blocks, NU_TILE, 0, s>>>(K, f, w, (const cd*)X, n, (cd*)g, (cd*)y);
  if (cudaGetLastError() != cudaSuccess) return TIKH_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? TIKH_OK : TIKH_ECUDA;
}
