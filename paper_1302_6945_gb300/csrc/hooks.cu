// hooks.cu -- test entry points of include/tikh.h that run one building block (the FFT engine, one
// leaf) on caller data, so that each stage can be compared with the CPU oracle on identical inputs.
#include <vector>

#include "internal.h"

using namespace tikh;

namespace tikh {

struct HookLoad {
  const cd* p;
  __device__ cd operator()(int, int64_t j) const { return p[j]; }
};
struct HookStore {
  cd* p;
  __device__ void operator()(int, int64_t k, cd v) const { p[k] = v; }
};

int launch_fft_test(int64_t L, cd* data, int sign, cudaStream_t s, int64_t* bytes_out) {
  Plan P;  // scratch plan holding only the twiddle tables
  P.stream = s;
  std::vector<void*> tmp;
  auto table = [&](int64_t n) -> cd* {
    cd* t = nullptr;
    if (cudaMalloc(&t, sizeof(cd) * (size_t)n) != cudaSuccess) return nullptr;
    tmp.push_back(t);
    launch_twiddle(t, n, s);
    return t;
  };
  FftPlan f;
  f.L = L;
  int rc = 0;
  if (L <= FFT_TILE_MAX) {
    if (!fft_factor((int)L, f.d1)) rc = TIKH_EINVAL;
    else f.d1.tw = table(L);
  } else {
    int64_t L1, L2;
    if (!fft_split(L, L1, L2)) rc = TIKH_EINVAL;
    else {
      f.four = true;
      f.L1 = L1;
      f.L2 = L2;
      fft_factor((int)L1, f.d1);
      fft_factor((int)L2, f.d2);
      f.d1.tw = table(L1);
      f.d2.tw = table(L2);
      f.twL = table(L);
    }
  }
  cd* work = nullptr;
  if (!rc && f.four && cudaMalloc(&work, sizeof(cd) * (size_t)L) != cudaSuccess) rc = TIKH_ENOMEM;
  if (work) tmp.push_back(work);
  if (!rc && fft_run(f, 1, sign, HookLoad{data}, HookStore{data}, work, s) < 0) rc = TIKH_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = TIKH_ECUDA;
  for (void* p : tmp) cudaFree(p);
  if (bytes_out) *bytes_out = 0;
  return rc;
}

}  // namespace tikh

extern "C" {

int tikh_test_fft(int64_t n, void* data, int sign, void* stream) {
  if (n < 1 || !data || (sign != 1 && sign != -1)) return TIKH_EINVAL;
  return launch_fft_test(n, (cd*)data, sign, (cudaStream_t)stream, nullptr);
}

int tikh_test_leaf(int K, const void* sigma, const void* r, const int* delta_in, double eps, void* B, int* len,
                   int* delta_out, int* order, int* pivot, int64_t* deferred, int* n_def, void* stream) {
  if (K < 1 || K > 64 || !sigma || !r || !delta_in || !B || !len || !delta_out || !order || !pivot || !deferred ||
      !n_def || !(eps >= 0.0))
    return TIKH_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int* st = nullptr;
  unsigned long long* colmax = nullptr;
  if (cudaMalloc(&st, sizeof(int) * 4) != cudaSuccess) return TIKH_ENOMEM;
  if (cudaMalloc(&colmax, sizeof(unsigned long long) * 8) != cudaSuccess) { cudaFree(st); return TIKH_ENOMEM; }
  cudaMemsetAsync(st, 0, sizeof(int) * 4, s);
  cudaMemsetAsync(n_def, 0, sizeof(int), s);
  cudaMemsetAsync(order, 0xff, sizeof(int) * K, s);
  cudaMemsetAsync(pivot, 0xff, sizeof(int) * K, s);
  cudaMemcpyAsync(delta_out, delta_in, sizeof(int) * 5, cudaMemcpyDeviceToDevice, s);
  int rc = launch_leaf_arrays(K, (const cd*)sigma, (const cd*)r, delta_out, eps, (cd*)B, len, colmax, n_def, deferred,
                              st, order, pivot, s);
  int hs = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = TIKH_ECUDA;
  else if (cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = TIKH_ECUDA;
  cudaFree(st);
  cudaFree(colmax);
  if (rc < 0) return rc;
  return hs ? TIKH_ENUMERIC : TIKH_OK;
}

}  // extern "C"
