// common.cuh -- complex FP64 helpers, device status bits and small utilities shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tikh {

using cd = double2;  // complex128 as (re, im)

__host__ __device__ __forceinline__ cd mkc(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ cd cadd(cd a, cd b) { return mkc(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return mkc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cmul(cd a, cd b) { return mkc(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)); }
// a * b + c
__device__ __forceinline__ cd cfma(cd a, cd b, cd c) {
  return mkc(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ cd cconj(cd a) { return mkc(a.x, -a.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return mkc(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(cd a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ bool cnonzero(cd a) { return a.x != 0.0 || a.y != 0.0; }

// device status word bits (plan->d_status)
enum : int {
  ST_NUMERIC = 1,    // final degree pattern wrong / zero pivot
  ST_DEGREE = 2,     // a basis degree exceeded the planned transform length
  ST_DIFFICULT = 4,  // deferred-condition list overflow
  ST_WAIT = 8,       // a bounded in-kernel wait gave up
  ST_INPUT = 16,     // a non-finite entry in col, row or the right-hand side
};

__device__ __forceinline__ void set_status(int* st, int bit) { atomicOr(st, bit); }

// twiddle exp(+2 pi i t / L) read from a table of length L (t reduced mod L by the caller)
__device__ __forceinline__ cd tw_at(const cd* __restrict__ tab, int64_t t) { return __ldg(tab + t); }

// Column scale carried with every basis: the consumer multiplies column j by 2^{-e_j} where
// colmax_j = f 2^{e_j}, f in [0.5, 1) (exact power-of-two scaling).
__device__ __forceinline__ double col_scale_from_bits(unsigned long long bits) {
  double mx = __longlong_as_double((long long)bits);
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);
  return ldexp(1.0, -e);
}

}  // namespace tikh
