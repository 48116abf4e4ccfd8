// noalloc.cu -- the FFT engine without any allocation: its scratch (the twiddle tables and the
// four-step temporary) lives in a file-scope device array of fixed size instead of cudaMalloc'd
// memory, for callers that must not allocate (see tikh_fft_noalloc in include/tikh.h).
#include <atomic>

#include "internal.h"

using namespace tikh;

namespace tikh {

// Largest transform length served.  Scratch layout (complex128 units):
//   [0, NA_MAX)                      twiddles of length n
//   [NA_MAX, NA_MAX + 2*FFT_TILE_MAX) twiddles of the two four-step factors
//   [.. , .. + NA_MAX)               four-step temporary
constexpr int64_t NA_MAX = 65536;
constexpr int64_t NA_SCRATCH = NA_MAX + 2 * FFT_TILE_MAX + NA_MAX;

static __device__ __align__(256) double2 g_noalloc_scratch[NA_SCRATCH];

struct NaLoad {
  const cd* p;
  __device__ cd operator()(int, int64_t j) const { return p[j]; }
};
struct NaStore {
  cd* p;
  __device__ void operator()(int, int64_t k, cd v) const { p[k] = v; }
};

// Device address of the scratch array for each device, fetched once with that device current.
// Host code cannot use the symbol itself as a device pointer.  Entries are atomic: host threads
// making their first call on the same device at once may both look the address up (the lookup
// returns the same value), but neither reads a torn or half-written entry.
static std::atomic<cd*> g_na_addr[64];

static int noalloc_scratch(cd** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return TIKH_ECUDA; }
  cd* a = g_na_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return TIKH_ECUDA; }
    a = (cd*)p;
    g_na_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return TIKH_OK;
}

}  // namespace tikh

extern "C" int tikh_fft_noalloc(int64_t n, void* data, int sign, void* stream) {
  if (n < 1 || !data || (sign != 1 && sign != -1)) return TIKH_EINVAL;
  if (n > NA_MAX) return TIKH_EINVAL;  // beyond the fixed scratch: use tikh_test_fft
  cd* scr = nullptr;
  int rc = noalloc_scratch(&scr);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  FftPlan f;
  f.L = n;
  cd* tw_n = scr;
  cd* tw_1 = scr + NA_MAX;
  cd* tw_2 = scr + NA_MAX + FFT_TILE_MAX;
  cd* tmp = scr + NA_MAX + 2 * FFT_TILE_MAX;
  // every call rewrites the tables it reads, so nothing depends on what an earlier call left behind
  if (n <= FFT_TILE_MAX) {
    if (!fft_factor((int)n, f.d1)) return TIKH_EINVAL;
    if (launch_twiddle(tw_n, n, s) < 0) return TIKH_ECUDA;
    f.d1.tw = tw_n;
  } else {
    int64_t L1, L2;
    if (!fft_split(n, L1, L2)) return TIKH_EINVAL;
    f.four = true;
    f.L1 = L1;
    f.L2 = L2;
    fft_factor((int)L1, f.d1);
    fft_factor((int)L2, f.d2);
    if (launch_twiddle(tw_n, n, s) < 0 || launch_twiddle(tw_1, L1, s) < 0 || launch_twiddle(tw_2, L2, s) < 0)
      return TIKH_ECUDA;
    f.d1.tw = tw_1;
    f.d2.tw = tw_2;
    f.twL = tw_n;
  }
  if (fft_run(f, 1, sign, NaLoad{(const cd*)data}, NaStore{(cd*)data}, tmp, s) < 0) return TIKH_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? TIKH_OK : TIKH_ECUDA;
}
