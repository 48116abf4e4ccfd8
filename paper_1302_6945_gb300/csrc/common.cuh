// common.cuh -- complex FP64 helpers, device status bits and small utilities shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

namespace tikh {

using cd = double2;  // complex128 as (re, im)
using cf = float2;   // complex64 as (re, im): the recursion's FFT stages in the FP32 precision pattern

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

// the same operations on complex64 (FP32 arithmetic, FP32 accumulation)
__host__ __device__ __forceinline__ cf mkcf(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ cf cadd(cf a, cf b) { return mkcf(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cf csub(cf a, cf b) { return mkcf(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cf cmul(cf a, cf b) { return mkcf(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
__device__ __forceinline__ cf cfma(cf a, cf b, cf c) {
  return mkcf(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ cf cconj(cf a) { return mkcf(a.x, -a.y); }
__device__ __forceinline__ cf cscale(cf a, float s) { return mkcf(a.x * s, a.y * s); }
__device__ __forceinline__ cd to_cd(cf a) { return mkc((double)a.x, (double)a.y); }
__device__ __forceinline__ cf to_cf(cd a) { return mkcf((float)a.x, (float)a.y); }

// generic construction and zero of either complex type
template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ cd czero<cd>() { return mkc(0.0, 0.0); }
template <> __device__ __forceinline__ cf czero<cf>() { return mkcf(0.0f, 0.0f); }
template <class C> __device__ __forceinline__ C cfrom(cd a);
template <> __device__ __forceinline__ cd cfrom<cd>(cd a) { return a; }
template <> __device__ __forceinline__ cf cfrom<cf>(cd a) { return to_cf(a); }

// Programmatic dependent launch.  The kernels of a solve form one long stream-ordered chain (about 65 000
// small launches for a c2 solve).  Launched with programmatic stream serialisation, a kernel lets its
// successor be scheduled as soon as all its own CTAs have started, and waits for its predecessor to finish
// (with its memory visible) before reading anything: the successor's launch latency overlaps the running
// kernel, while every kernel still sees all of its predecessors' writes (each one waits for its predecessor,
// which itself waited for its own).  Without the launch attribute both instructions do nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// whether solves launch their chain kernels with programmatic serialisation: only when the environment
// variable TIKH_PDL is "1" (read once per process)
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("TIKH_PDL");
    return v && v[0] == '1';
  }();
  return on;
}

// launch kernel k with or without programmatic stream serialisation
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

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
__device__ __forceinline__ cf tw_at(const cf* __restrict__ tab, int64_t t) { return __ldg(tab + t); }

// Column scale carried with every basis: the consumer multiplies column j by 2^{-e_j} where
// colmax_j = f 2^{e_j}, f in [0.5, 1) (exact power-of-two scaling).
__device__ __forceinline__ double col_scale_from_bits(unsigned long long bits) {
  double mx = __longlong_as_double((long long)bits);
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);
  return ldexp(1.0, -e);
}

// The same scale as an exponent k (scale = 2^k) by integer operations on the bit pattern: a normal column
// maximum with biased exponent E in [1, 2044] has frexp exponent E - 1022, so k = 1022 - E.  ok = false for
// a zero, sub-normal or near-overflow maximum (then col_scale_from_bits applies).
__device__ __forceinline__ int col_shift_from_bits(unsigned long long bits, bool& ok) {
  const int E = (int)(bits >> 52);  // a non-negative double: no sign bit
  ok = E >= 1 && E <= 2044;
  return 1022 - E;
}

// v 2^k for k in [-1022, 1021], exactly as the FP64 multiply by 2^k rounds it: an add to the exponent field
// (no FP64 instruction) when v and the result are normal; zeros unchanged; otherwise the multiply
__device__ __forceinline__ double mul_pow2(double v, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ULL) return v;
  const int e = (int)((b >> 52) & 0x7ffULL);
  if (e == 0 || e == 2047 || e + k <= 0 || e + k >= 2047)
    return v * __longlong_as_double((long long)(1023 + k) << 52);
  return __longlong_as_double((long long)(b + ((unsigned long long)(long long)k << 52)));
}
__device__ __forceinline__ cd cmul_pow2(cd v, int k) { return mkc(mul_pow2(v.x, k), mul_pow2(v.y, k)); }

// v times the column scale of a column maximum's bit pattern (col_scale_from_bits), exact
__device__ __forceinline__ cd col_scaled(cd v, unsigned long long bits) {
  bool ok;
  const int k = col_shift_from_bits(bits, ok);
  return ok ? cmul_pow2(v, k) : cscale(v, col_scale_from_bits(bits));
}

}  // namespace tikh
