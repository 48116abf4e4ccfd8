// leaf.cu -- leaves of Algorithm 1: the serial single-point construction of Eq. (spbasis) over the
// K = 2 NS L conditions of a leaf node (K <= 64 for the 5 x 5 basis of the l2 and Toeplitz-Gramian
// problems, K <= 42 for the 7 x 7 basis of the general problem), with condition pivoting (Sec. 5) and
// difficult-point deferral; and the end-of-run serial processing of the deferred conditions against B*.
//
// Pivot rules (shared reading of the paper):
//  - pivot column of a condition: minimum current tau-degree among its non-zero residual entries;
//    ties: larger |r|^2, then lower column index;
//  - next condition: largest |r_pivot|^2 / ||r||^2; ties: lowest list position (2 NS j + NS c + f);
//  - if that best ratio is below eps^2, the leaf's remaining conditions are deferred.
// Decisions are taken in FP64 values; the comparisons use the IEEE bit patterns of the non-negative
// doubles as integers (same order, no FP64 instruction).
//
// Cost model on GB300: an FP64 warp instruction occupies its SM sub-partition for 64 cycles whatever
// the number of active lanes (measured), FP32 ~4.5 cycles.  The pivot chain of a leaf therefore keeps
// only the FP64 work that decides the next step (scores, the multipliers mu, the residual update), and
// spreads each residual row over W lanes ("component lanes") so that the per-entry work of a step
// is one warp instruction on each of the four sub-partitions; the basis B_leaf = E_1 E_2 ... E_K is
// rebuilt by four more warps from the recorded (pivot, sigma, mu) of each step as soon as the chain
// publishes it.
#include "internal.h"

namespace tikh {

// leaf sizes by basis size W: conditions per leaf, stored coefficients per entry, residual rows per
// chain warp (W lanes each)
template <int W>
struct LeafDims {
  static constexpr int KMAX = W == 5 ? 64 : 42;
  static constexpr int CAP = KMAX + 1;
  static constexpr int RPW = 32 / W;
};
constexpr int LEAF_KMAX = 64;  // the largest over W
constexpr int LEAF_SPIN_DEFAULT = 1 << 24;  // polls of the rebuild warps before they give up (ST_WAIT)

// pick: (score bits, position, pivot); larger score wins, then lower position
struct Pick {
  unsigned long long sb;
  int idx, piv;
};
__device__ __forceinline__ bool pick_better(const Pick& b, const Pick& a) {
  return b.sb > a.sb || (b.sb == a.sb && b.idx < a.idx);
}
__device__ __forceinline__ Pick warp_pick(Pick p) {
  for (int o = 16; o > 0; o >>= 1) {
    Pick q;
    q.sb = __shfl_xor_sync(0xffffffffu, p.sb, o);
    q.idx = __shfl_xor_sync(0xffffffffu, p.idx, o);
    q.piv = __shfl_xor_sync(0xffffffffu, p.piv, o);
    if (pick_better(q, p)) p = q;
  }
  return p;
}
constexpr unsigned long long NO_PICK = 0ULL;  // every real score bit pattern is > 0 (score > 0)

// non-zero test on the bit pattern (no FP64 instruction): +0.0 and -0.0 are zero
__device__ __forceinline__ bool nz_bits(double v) { return ((unsigned long long)__double_as_longlong(v) << 1) != 0ULL; }
__device__ __forceinline__ bool cnz(cd a) { return nz_bits(a.x) || nz_bits(a.y); }

// sum of the W magnitudes in a fixed order (pairs, then the pair sums, then the odd one)
template <int W>
__device__ __forceinline__ double mag_sum(const double* m) {
  if (W == 5) return ((m[0] + m[1]) + (m[2] + m[3])) + m[4];
  return (((m[0] + m[1]) + (m[2] + m[3])) + (m[4] + m[5])) + m[W - 1];
}
template <int W>
__device__ __forceinline__ float mag_sum_f(const float* m) {
  if (W == 5) return ((m[0] + m[1]) + (m[2] + m[3])) + m[4];
  return (((m[0] + m[1]) + (m[2] + m[3])) + (m[4] + m[5])) + m[W - 1];
}

// pivot column and score of one residual row (score > 0 for a row with a non-zero entry)
template <int W>
__device__ __forceinline__ Pick score_row(const cd* r, const int* dl, int q) {
  unsigned long long mb[W];
  double mag[W], tot;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    mag[i] = fma(r[i].x, r[i].x, r[i].y * r[i].y);
    mb[i] = (unsigned long long)__double_as_longlong(mag[i]);
  }
  tot = mag_sum<W>(mag);
  int pi = -1;
  unsigned long long mpi = 0ULL;
  double magpi = 0.0;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    if (!cnz(r[i])) continue;
    if (pi < 0 || dl[i] < dl[pi] || (dl[i] == dl[pi] && mb[i] > mpi)) { pi = i; mpi = mb[i]; magpi = mag[i]; }
  }
  Pick p;
  p.idx = q;
  p.piv = pi;
  p.sb = NO_PICK;
  if (pi >= 0) {
    double sc = magpi / tot;
    p.sb = (unsigned long long)__double_as_longlong(sc);
    if (p.sb == 0ULL) p.sb = 1ULL;  // an underflowed ratio still ranks above "no candidate"
  }
  return p;
}

// degree bound of entry (i, j) of a node basis: tau-degree bound for pivoted columns, accumulation
// bound (largest pivoted delta_out - delta_in_i) for the others, diagonal >= 0
template <int W>
__device__ __forceinline__ int entry_bound(const int* din, const int* dout, int i, int j) {
  int amax = 0;
  bool have = false;
  for (int c = 0; c < W; ++c)
    if (dout[c] > din[c]) { amax = have ? max(amax, dout[c]) : dout[c]; have = true; }
  if (dout[j] > din[j]) return dout[j] - din[i];
  int acc = have ? amax - din[i] : -1;
  if (i == j && acc < 0) acc = 0;
  return min(acc, dout[j] - din[i]);
}

// condition source of a leaf: the recursion node (a, s, L) in problem pb's residual rows (NS rows of W
// entries per node), with position q = 2 NS j + NS c + f <-> node e = a + c + s j, condition f; deferred
// ids are NS e + f
template <int W, int NS>
struct SrcNodes {
  const cd* R;
  const cd* wN;
  int64_t N, a, s;
  __device__ void get1(int pb, int q, int jcol, cd& rj, cd& sig, int64_t& id) const {
    int j = q / (2 * NS), c = (q / NS) % 2, f = q % NS;
    int64_t e = a + c + s * j;
    id = NS * e + f;
    rj = R[((int64_t)pb * N + e) * (NS * W) + f * W + jcol];
    sig = wN[e];
  }
};
// explicit arrays (test hook, one problem, 5 x 5 basis): sigma[q], r[5q..5q+4]; deferred ids are q
struct SrcArrays {
  const cd* sigma;
  const cd* rr;
  __device__ void get1(int, int q, int jcol, cd& rj, cd& sig, int64_t& id) const {
    id = q;
    rj = rr[q * 5 + jcol];
    sig = sigma[q];
  }
};

__device__ __forceinline__ cd shfl_cd(cd v, int src) {
  return mkc(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// One CTA per problem (blockIdx.x), "component lanes": with RPW = 32 / W rows per warp, chain warp w holds
// residual rows RPW w .. RPW w + RPW - 1, lane W rr + j holding entry j of row RPW w + rr (6 rows and lanes
// 30, 31 idle for W = 5; 4 rows and lanes 28-31 idle for W = 7), so the FP64 work of a step that is per entry
// (magnitudes, the update) is one warp instruction spread over CWN warps on all four SM sub-partitions.
// Each step: magnitudes -> row scores (every lane of a row gathers its W
// magnitudes) -> per-warp pick -> one named barrier among the chain warps -> the same global pick in
// every chain warp -> multipliers mu_j (lane j's own column) -> update.  Chain warp 0 publishes the
// records of step s and then the count s + 1; the four rebuild warps (one per sub-partition) apply
// B <- B E_s as soon as step s is published, so the chain never waits for the rebuild.
constexpr long long KEY_NONE = -0x7fffffffffffffffLL - 1;
constexpr long long KEY_BAND = 16;  // units of 2^-23 in log2 scale; the key's error is below 8 units
constexpr long long KEY_SPEC = 0x7fffffffffffffffLL;  // a warp holding a special row (FP64 path)

// Approximate key of the row score |r_pi|^2 / ||r||^2 from the exact FP64 magnitudes' bit patterns,
// in FP32 and integer arithmetic: key = 2^23 (floor(log2 R) + 127) + (23 leading mantissa bits of R),
// monotone in R.  Magnitudes are re-based to the row's largest exponent (terms more than 2^60 below it
// are dropped), truncated to 23 mantissa bits, summed in FP32 and divided to 2 ulp, so the key is
// within 8 units of the exact ratio's (W - 1 <= 6 additions); two keys more than KEY_BAND apart order
// the FP64 scores the same way.  special: zero
// or sub-normal pivot magnitude, or a row too small or too large for the re-basing (FP64 path instead).
template <int W>
__device__ __forceinline__ long long approx_key(const double* mg, unsigned long long mpi, bool& special) {
  unsigned long long mb[W];
  int emax = 0;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    mb[c] = (unsigned long long)__double_as_longlong(mg[c]);
    emax = max(emax, (int)(mb[c] >> 52));
  }
  const int epi = (int)(mpi >> 52);
  special = epi == 0 || emax <= 61 || emax >= 2046;
  float f[W];
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const int ec = (int)(mb[c] >> 52), d = ec - emax;
    f[c] = (d < -60 || ec == 0) ? 0.0f : __int_as_float(((127 + d) << 23) | (int)((mb[c] >> 29) & 0x7fffffULL));
  }
  const float tot = mag_sum_f<W>(f);  // in [1, 2 W)
  const float mp = __int_as_float((127 << 23) | (int)((mpi >> 29) & 0x7fffffULL));  // in [1, 2)
  const float qf = __fdividef(mp, tot);  // normal, in (1 / (2 W), 2); within 2 ulp
  return ((long long)(epi - emax) << 23) + (long long)__float_as_int(qf);
}

// 1/d for a positive normal d with biased exponent in (2, 2044): seed y0 from the FP32 approximate
// reciprocal of d's 23 leading mantissa bits (relative error e0 below 2^-21), then one third-order
// step of the series 1/d = y0 / (1 - e) = y0 (1 + e + e^2 + ...), e = 1 - d y0: the truncation error
// e^3 is below 2^-63, under FP64 rounding
__device__ __forceinline__ double rcp_series(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int E = (int)(b >> 52);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__int_as_float((127 << 23) | (int)((b >> 29) & 0x7fffffULL))));
  const int fb = __float_as_int(rf);  // rf in [0.5, 1]
  const long long ye = (long long)(((fb >> 23) - 127) - (E - 1023) + 1023);
  const double y = __longlong_as_double((long long)(((unsigned long long)ye << 52) | ((unsigned long long)(fb & 0x7fffff) << 29)));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// test hook: rcp_series on an array of positive normal doubles (biased exponent in (2, 2044))
__global__ void k_test_rcp(const double* __restrict__ d, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rcp_series(d[i]);
}

int launch_rcp_test(const double* d, double* out, int64_t n, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  k_test_rcp<<<blocks, 256, 0, s>>>(d, out, n);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

constexpr int L4_NREC = 128;
constexpr int CHAIN_DONE = 1 << 30;

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ void st_volatile(int* p, int v) { *(volatile int*)p = v; }

template <int W, int CWN, class Src>
__global__ void __launch_bounds__(32 * CWN + L4_NREC, CWN <= 4 ? 4 : (CWN <= 8 ? 2 : 1)) k_leaf(Src src, int K, int* delta, int* dstack,
                                                              unsigned long long save_mask, double eps, BasisBuf out,
                                                              int* ndiff, int64_t* diff, int maxdiff, int* status,
                                                              int* rec_order, int* rec_pivot, const int* bad,
                                                              int spin_limit) {
  constexpr int NCHAIN = 32 * CWN, NT = NCHAIN + L4_NREC;
  constexpr int WW = W * W, KMAX = LeafDims<W>::KMAX, CAP = LeafDims<W>::CAP, RPW = LeafDims<W>::RPW;
  __shared__ cd Bs[WW][CAP];
  __shared__ cd oldc[W][CAP];
  __shared__ int rec_w[KMAX], rec_piv[KMAX];  // winner row and pivot column of each step
  __shared__ cd muspec[KMAX][W];  // each active row's would-be multipliers; a row is written only
                                  // while it is active, so a step's winner row stays as it was
  __shared__ cd sigbuf[KMAX];
  __shared__ longlong2 cand2[2][CWN];  // per-warp two largest packed keys ((key * 64 + 63 - row) * 8 +
                                      // pivot column; KEY_SPEC: a special row), by step parity
  __shared__ Pick cand[2][CWN];    // per-warp exact picks (FP64 path), by step parity
  __shared__ int blen[WW];
  __shared__ int din[W], dl_out[W];
  __shared__ int chain_state;  // steps recorded so far, | CHAIN_DONE once the chain has stopped
  __shared__ int rb_cmd;
  pdl_enter();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, pb = blockIdx.x;
  int* dlt = delta + DSTR * pb;

  if (tid < W) din[tid] = dlt[tid];
  if (tid == 0) chain_state = 0;
  if (tid < WW) blen[tid] = (tid % (W + 1) == 0) ? 1 : 0;
  for (int idx = tid; idx < WW * CAP; idx += NT) {
    int e = idx / CAP, t = idx % CAP;
    Bs[e][t] = (t == 0 && e % (W + 1) == 0) ? mkc(1.0, 0.0) : mkc(0.0, 0.0);
  }
  const int rr = lane / W, jc = lane - W * rr, rbase = W * rr;
  const int q = wid * RPW + rr;
  // a problem whose input failed the prologue's finiteness check processes no condition
  const bool skip = bad && bad[pb] != 0;
  bool active = tid < NCHAIN && rr < RPW && q < K && !skip;
  cd r = mkc(0.0, 0.0), sig = mkc(0.0, 0.0);
  int64_t eid = -1;
  if (active) {
    src.get1(pb, q, jc, r, sig, eid);
    if (jc == 0) sigbuf[q] = sig;
  }
  __syncthreads();
  if (tid < W && dstack) {
    for (int d = 0; d < MAX_DEPTH; ++d)
      if (save_mask >> d & 1ULL) dstack[((int64_t)pb * MAX_DEPTH + d) * DSTR + tid] = din[tid];
  }

  if (tid < NCHAIN) {
    int dl[W];  // tau-degrees of the W columns, identical in every chain lane
#pragma unroll
    for (int i = 0; i < W; ++i) dl[i] = din[i];
    const unsigned long long eps_bits = (unsigned long long)__double_as_longlong(eps * eps);
    // eps^2 as a key (the same scale as approx_key); for zero or sub-normal eps^2 the key of 2^-1022
    const int eexp = (int)(eps_bits >> 52);
    const bool eps_normal = eexp > 0 && eexp < 2047;
    const long long key_eps = eps_normal ? ((long long)(eexp - 1023 + 127) << 23) + (long long)((eps_bits >> 29) & 0x7fffffULL)
                                         : ((long long)(-1022 + 127) << 23);
    for (int step = 0;; ++step) {
      const int par = step & 1;
      // ---- score of every active row (same arithmetic as the row-per-lane form) ----
      const double mag = fma(r.x, r.x, r.y * r.y);
      const unsigned nzm = __ballot_sync(0xffffffffu, active && cnz(r));
      const unsigned rownz = (nzm >> rbase) & ((1u << W) - 1u);
      double mg[W];
#pragma unroll
      for (int c = 0; c < W; ++c) mg[c] = __shfl_sync(0xffffffffu, mag, (rbase + c) & 31);
      if (active && rownz == 0u) active = false;  // every entry zero: the condition already holds
      // the row's pivot column, in each of its W lanes
      int rpi = -1, dpi = 0;
      unsigned long long mpi = 0ULL;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (!((rownz >> c) & 1u)) continue;
        const unsigned long long mb = (unsigned long long)__double_as_longlong(mg[c]);
        if (rpi < 0 || dl[c] < dpi || (dl[c] == dpi && mb > mpi)) { rpi = c; mpi = mb; dpi = dl[c]; }
      }
      // the multipliers this row would give if it wins, mu_j = -r_j conj(r_pi) / |r_pi|^2 (lane j's
      // column), computed before the pick so that their FP64 latency overlaps the pick's integer work
      const cd rpr = shfl_cd(r, (rbase + max(rpi, 0)) & 31);
      {
        const int de = (int)(mpi >> 52);
        const double dw = __longlong_as_double((long long)mpi);  // |r_pi|^2 exactly as scored
        const bool slow = active && !(de > 2 && de < 2044);
        double rd = rcp_series(dw);
        if (__any_sync(0xffffffffu, slow)) {  // zero, sub-normal or extreme |r_pi|^2: the FP64 division
          if (slow) rd = 1.0 / dw;
        }
        // r_j conj(r_pi) does not wait for the reciprocal
        const cd t = mkc(fma(r.x, rpr.x, r.y * rpr.y), fma(r.y, rpr.x, -(r.x * rpr.y)));
        if (active && jc != rpi) muspec[q][jc] = mkc(-(t.x * rd), -(t.y * rd));
      }
      long long p1 = KEY_NONE, p2 = KEY_NONE;
      if (active && jc == 0) {
        bool spec;
        p1 = (approx_key<W>(mg, mpi, spec) * 64 + (63 - q)) * 8 + rpi;
        if (spec) p1 = KEY_SPEC;
      }
      // the two largest over the candidate lanes 0, W, ..., (RPW - 1) W (the result in lane 0)
#pragma unroll
      for (int o = W; o < RPW * W; o *= 2) {
        long long a1 = __shfl_down_sync(0xffffffffu, p1, o), a2 = __shfl_down_sync(0xffffffffu, p2, o);
        if (lane + o >= 32) { a1 = KEY_NONE; a2 = KEY_NONE; }
        const long long hi = max(p1, a1), lo = min(p1, a1);
        p2 = max(lo, max(p2, a2));
        p1 = hi;
      }
      if (lane == 0) cand2[par][wid] = make_longlong2(p1, p2);
      named_sync(2, NCHAIN);
      long long g1 = KEY_NONE, g2 = KEY_NONE;
#pragma unroll
      for (int w2 = 0; w2 < CWN; ++w2) {
        const longlong2 c = cand2[par][w2];
        const long long hi = max(g1, c.x), lo = min(g1, c.x);
        g2 = max(lo, max(g2, c.y));
        g1 = hi;
      }
      bool exact = g1 == KEY_SPEC;
      if (!exact && g1 != KEY_NONE) {
        const long long k1 = g1 >> 9;
        if (g2 != KEY_NONE && k1 - (g2 >> 9) <= KEY_BAND) exact = true;  // a near tie
        if (k1 <= key_eps + KEY_BAND && (k1 >= key_eps - KEY_BAND || !eps_normal)) exact = true;
      }
      int outcome, w = -1, pi = -1;  // outcome 0: pivot step, 1: no condition left, 2: difficult
      if (!exact) {
        if (g1 == KEY_NONE) {
          outcome = 1;
        } else {
          w = 63 - (int)((g1 >> 3) & 63);
          pi = (int)(g1 & 7);
          outcome = (g1 >> 9) < key_eps ? 2 : 0;
        }
      } else {  // FP64 scores of every candidate, as the approximate keys could not decide
        Pick p;
        p.sb = NO_PICK;
        p.idx = 1 << 30;
        p.piv = -1;
        if (active && jc == 0) {
          const double tot = mag_sum<W>(mg);
          const double sc = __longlong_as_double((long long)mpi) / tot;
          p.sb = (unsigned long long)__double_as_longlong(sc);
          if (p.sb == 0ULL) p.sb = 1ULL;  // an underflowed ratio still ranks above "no candidate"
          p.idx = q;
          p.piv = rpi;
        }
        p = warp_pick(p);
        if (lane == 0) cand[par][wid] = p;
        named_sync(2, NCHAIN);
        Pick b = cand[par][0];
#pragma unroll
        for (int w2 = 1; w2 < CWN; ++w2)
          if (pick_better(cand[par][w2], b)) b = cand[par][w2];
        outcome = b.sb == NO_PICK ? 1 : (b.sb < eps_bits ? 2 : 0);
        w = b.idx;
        pi = b.piv;
      }
      if (outcome != 0) {  // done, or difficult: defer the rest of the leaf
        if (outcome == 2 && active && jc == 0) {
          int slot = atomicAdd(ndiff + 4 * pb, 1);
          if (slot < maxdiff) diff[(int64_t)pb * maxdiff + slot] = eid;
          else set_status(status, ST_DIFFICULT);
        }
        if (tid == 0) {
          __threadfence_block();
          st_volatile(&chain_state, step | CHAIN_DONE);
        }
        break;
      }
      const cd sw = sigbuf[w];
      const cd muw = muspec[w][jc];
      if (tid == 0) {  // this step's record, then its publication to the rebuild warps
        rec_w[step] = w;
        rec_piv[step] = pi;
        if (rec_order) { rec_order[step] = w; rec_pivot[step] = pi; }
        __threadfence_block();
        st_volatile(&chain_state, step + 1);
      }
      if (q == w) active = false;
#pragma unroll
      for (int c = 0; c < W; ++c) dl[c] += (c == pi) ? 1 : 0;
      // ---- r <- r E(sigma): column pi times (sigma - sw), the others += mu_j r_pi ----
      const cd rpo = shfl_cd(r, (rbase + pi) & 31);
      if (active) {
        const cd ds = csub(sig, sw);
        const cd fac = (jc == pi) ? ds : muw;
        const cd base = (jc == pi) ? mkc(0.0, 0.0) : r;
        r = cfma(fac, rpo, base);
      }
    }
    if (tid < W) dl_out[tid] = dl[tid];
  } else {
    // ---- rebuild B <- B E_s for s = 0, 1, ... as the chain publishes them ----
    const int rt = tid - NCHAIN;
    for (int s = 0;; ++s) {
      if (rt == 0) {
        int cmd = 2;  // 0: step s is recorded, 1: the chain stopped before s, 2: gave up waiting
        for (int it = 0; it < spin_limit; ++it) {
          const int st = ld_volatile(&chain_state);
          if ((st & ~CHAIN_DONE) > s) { cmd = 0; break; }
          if (st & CHAIN_DONE) { cmd = 1; break; }
          __nanosleep(20);
        }
        __threadfence_block();
        if (cmd == 2) set_status(status, ST_WAIT);
        rb_cmd = cmd;
      }
      named_sync(1, L4_NREC);
      if (rb_cmd != 0) break;
      const int pi = rec_piv[s], ws = rec_w[s];
      const cd sb = sigbuf[ws];
      const cd nsb = mkc(-sb.x, -sb.y);
      int lmax = 0;
#pragma unroll
      for (int i = 0; i < W; ++i) lmax = max(lmax, blen[i * W + pi]);
      for (int idx = rt; idx < W * lmax; idx += L4_NREC) {
        int i = idx / lmax, t = idx % lmax;
        oldc[i][t] = Bs[i * W + pi][t];
      }
      named_sync(1, L4_NREC);
      // item (entry e = (i, j), coefficient t): column pi <- (z - sb) column pi, column j += mu_j old pi
      for (int idx = rt; idx < WW * (lmax + 1); idx += L4_NREC) {
        const int e = idx / (lmax + 1), t = idx % (lmax + 1);
        const int i = e / W, j = e % W;
        const int lo = blen[i * W + pi];
        if (lo == 0 || t > lo) continue;
        const bool isp = j == pi;
        if (!isp && t == lo) continue;
        const cd o = t < lo ? oldc[i][t] : mkc(0.0, 0.0);
        const cd fac = isp ? nsb : muspec[ws][j];
        const cd base = isp ? (t >= 1 ? oldc[i][t - 1] : mkc(0.0, 0.0)) : Bs[e][t];
        Bs[e][t] = cfma(fac, o, base);
      }
      named_sync(1, L4_NREC);
      if (rt < W) {
        int i = rt, lo = blen[i * W + pi];
        if (lo > 0) {
          for (int j = 0; j < W; ++j)
            if (j != pi && blen[i * W + j] < lo) blen[i * W + j] = lo;
          blen[i * W + pi] = lo + 1;
        }
      }
      // the next poll's barrier orders these blen writes before the next step reads them
    }
  }
  __syncthreads();
  // ---- trim to the degree bounds, record column maxima, write out ----
  __shared__ unsigned long long cmax[W];
  if (tid < W) cmax[tid] = 0ULL;
  if (tid < WW) {
    int i = tid / W, j = tid % W;
    int bnd = entry_bound<W>(din, dl_out, i, j);
    int want = bnd < 0 ? 0 : bnd + 1;
    if (blen[tid] > want) blen[tid] = want;
  }
  __syncthreads();
  cd* oc = out.cp(pb);
  for (int idx = tid; idx < WW * CAP; idx += NT) {
    int e = idx / CAP, t = idx % CAP;
    if (t < blen[e]) {
      cd v = Bs[e][t];
      oc[(int64_t)e * out.cap + t] = v;
      double m = fmax(fabs(v.x), fabs(v.y));
      if (m > 0.0) atomicMax(&cmax[e % W], (unsigned long long)__double_as_longlong(m));
    }
  }
  __syncthreads();
  if (tid < WW) out.lp(pb)[tid] = blen[tid];
  if (tid < W) {
    out.mp(pb)[tid] = cmax[tid];
    dlt[tid] = dl_out[tid];
  }
}

template <int W, class Src>
static int launch_leaf_t(const Src& src, int K, int nb, int* delta, int* dstack, unsigned long long mask, double eps,
                         const BasisBuf& out, int* ndiff, int64_t* diff, int maxdiff, int* status, int* order,
                         int* pivot, const int* bad, int spin_limit, cudaStream_t s) {
  constexpr int RPW = LeafDims<W>::RPW;
  if (K > LeafDims<W>::KMAX) return TIKH_EINVAL;
  if (K <= 4 * RPW)
    launch_k(pdl_enabled(), k_leaf<W, 4, Src>, dim3(nb), dim3(32 * 4 + L4_NREC), 0, s, src, K, delta, dstack, mask, eps, out, ndiff, diff, maxdiff, status, order, pivot, bad, spin_limit);
  else if (K <= 8 * RPW)
    launch_k(pdl_enabled(), k_leaf<W, 8, Src>, dim3(nb), dim3(32 * 8 + L4_NREC), 0, s, src, K, delta, dstack, mask, eps, out, ndiff, diff, maxdiff, status, order, pivot, bad, spin_limit);
  else
    launch_k(pdl_enabled(), k_leaf<W, 11, Src>, dim3(nb), dim3(32 * 11 + L4_NREC), 0, s, src, K, delta, dstack, mask, eps, out, ndiff, diff, maxdiff, status, order, pivot, bad, spin_limit);
  return cudaGetLastError() == cudaSuccess ? 1 : TIKH_ECUDA;
}

int launch_leaf(Plan& P, const Step& st) {
  const int K = (int)(2 * P.ns * st.L);
  if (P.w == 7)
    return launch_leaf_t<7>(SrcNodes<7, 3>{P.R, P.wN, P.N, st.a, st.s}, K, P.nb, P.delta, P.dstack, st.save_mask,
                            P.opts.eps_diff, P.buf[st.depth][st.side], P.ndiff, P.diff, P.opts.max_difficult,
                            P.status, nullptr, nullptr, P.bad, P.wait_polls, P.stream);
  return launch_leaf_t<5>(SrcNodes<5, 2>{P.R, P.wN, P.N, st.a, st.s}, K, P.nb, P.delta, P.dstack, st.save_mask,
                          P.opts.eps_diff, P.buf[st.depth][st.side], P.ndiff, P.diff, P.opts.max_difficult, P.status,
                          nullptr, nullptr, P.bad, P.wait_polls, P.stream);
}

// test hook: one leaf (one problem) on explicit device arrays
int launch_leaf_arrays(int K, const cd* sigma, const cd* r, int* delta, double eps, cd* B, int* len,
                       unsigned long long* colmax, int* ndiff, int64_t* diff, int* status, int* order, int* pivot,
                       cudaStream_t s) {
  if (K < 1 || K > LEAF_KMAX) return TIKH_EINVAL;
  BasisBuf out;
  out.c = B;
  out.len = len;
  out.colmax = colmax;
  out.cap = K + 1;
  return launch_leaf_t<5>(SrcArrays{sigma, r}, K, 1, delta, nullptr, 0ULL, eps, out, ndiff, diff, K, status, order,
                          pivot, nullptr, LEAF_SPIN_DEFAULT, s);
}

// ------------------------------------------------------------------------------------------------
// difficult points (Sec. 5): residual against the final basis B*, then serial processing.
// ------------------------------------------------------------------------------------------------

// B*(sigma_q) for every deferred condition q (column scales applied): block (entry E, slot, problem),
// threads over the coefficients with the twiddle index advanced incrementally, a block reduction per q
template <int W, int NS>
__global__ void __launch_bounds__(256) k_diff_values(BasisBuf B, const cd* __restrict__ wN, int64_t N,
                                                     const int* ndiff, const int64_t* diff, int maxdiff, cd* vals) {
  __shared__ cd red[8];
  const int E = blockIdx.x, pb = blockIdx.z, tid = threadIdx.x;
  const int nd = min(ndiff[4 * pb], maxdiff);
  const cd* bc = B.cp(pb) + (int64_t)E * B.cap;
  const int64_t L = B.lp(pb)[E];
  const double scl = col_scale_from_bits(B.mp(pb)[E % W]);
  for (int q = blockIdx.y; q < nd; q += gridDim.y) {
    const int64_t e = diff[(int64_t)pb * maxdiff + q] / NS;
    int64_t ix = (e * (int64_t)tid) % N;
    const int64_t stp = (e * (int64_t)blockDim.x) % N;
    cd acc = mkc(0.0, 0.0);
    for (int64_t t = tid; t < L; t += blockDim.x) {
      acc = cfma(bc[t], tw_at(wN, ix), acc);
      ix += stp;
      if (ix >= N) ix -= N;
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      cd sum = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) sum = cadd(sum, red[w]);
      vals[((int64_t)pb * maxdiff + q) * (W * W) + E] = cscale(sum, scl);
    }
    __syncthreads();
  }
}

// r_q = Phi_q B*(sigma_q): thread per (deferred condition, column)
template <int W, int NS>
__global__ void k_diff_rows(const cd* __restrict__ Phi, int64_t N, const int* ndiff, const int64_t* diff, int maxdiff,
                            const cd* __restrict__ vals, cd* diffr) {
  const int pb = blockIdx.y;
  const int nd = min(ndiff[4 * pb], maxdiff);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < W * nd; idx += gridDim.x * blockDim.x) {
    const int q = idx / W, j = idx % W;
    const int64_t id = diff[(int64_t)pb * maxdiff + q], e = id / NS, f = id % NS;
    const cd* v = vals + ((int64_t)pb * maxdiff + q) * (W * W);
    cd acc = mkc(0.0, 0.0);
    for (int i = 0; i < W; ++i) acc = cfma(Phi[((int64_t)pb * N + e) * (NS * W) + f * W + i], v[i * W + j], acc);
    diffr[((int64_t)pb * maxdiff + q) * W + j] = acc;
  }
}

template <int W, int NS>
__global__ void __launch_bounds__(1024) k_diff_serial(BasisBuf B, const cd* __restrict__ wN, const int* ndiff,
                                                     const int64_t* diff, int maxdiff, cd* diffr, int* delta,
                                                     int* status, cd* scratch, int64_t scr_stride) {
  constexpr int WW = W * W;
  __shared__ int dl[W];
  __shared__ Pick wpick[32];
  __shared__ Pick best;
  __shared__ cd mu[W];
  __shared__ int blen[WW];
  __shared__ double scl[W];
  const int pb = blockIdx.x;
  const int nd = min(ndiff[4 * pb], maxdiff);
  if (nd == 0) return;
  const int tid = threadIdx.x;
  cd* bc = B.cp(pb);
  cd* scr = scratch + (int64_t)pb * scr_stride;
  cd* dr = diffr + (int64_t)pb * maxdiff * W;
  const int64_t* did = diff + (int64_t)pb * maxdiff;
  int* dlt = delta + DSTR * pb;
  if (tid < W) { dl[tid] = dlt[tid]; scl[tid] = col_scale_from_bits(B.mp(pb)[tid]); }
  if (tid < WW) blen[tid] = B.lp(pb)[tid];
  __syncthreads();
  // materialise the column scales so that B* is plain
  for (int E = 0; E < WW; ++E)
    for (int64_t t = tid; t < blen[E]; t += blockDim.x) bc[E * B.cap + t] = cscale(bc[E * B.cap + t], scl[E % W]);
  __syncthreads();
  unsigned char* done = (unsigned char*)(scr + W * B.cap);  // nd flags
  for (int q = tid; q < nd; q += blockDim.x) done[q] = 0;
  __syncthreads();
  for (int step = 0; step < nd; ++step) {
    Pick p;
    p.sb = NO_PICK; p.idx = 1 << 30; p.piv = -1;
    for (int q = tid; q < nd; q += blockDim.x) {
      if (done[q]) continue;
      Pick c = score_row<W>(dr + (int64_t)q * W, dl, q);
      if (c.piv < 0) { done[q] = 1; continue; }
      if (pick_better(c, p)) p = c;
    }
    p = warp_pick(p);
    if ((tid & 31) == 0) wpick[tid >> 5] = p;
    __syncthreads();
    if (tid == 0) {
      Pick b = wpick[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (pick_better(wpick[w], b)) b = wpick[w];
      best = b;
      if (b.sb != NO_PICK) {
        const cd* rs = dr + (int64_t)b.idx * W;
        int pi = b.piv;
        double den = rs[pi].x * rs[pi].x + rs[pi].y * rs[pi].y;
        cd inv = mkc(rs[pi].x / den, -rs[pi].y / den);
        for (int i = 0; i < W; ++i) {
          cd m = (i == pi) ? mkc(0.0, 0.0) : cmul(rs[i], inv);
          mu[i] = mkc(-m.x, -m.y);
        }
        done[b.idx] = 1;
      }
    }
    __syncthreads();
    const Pick b = best;
    if (b.sb == NO_PICK) break;
    const int pi = b.piv;
    const cd sb = tw_at(wN, did[b.idx] / NS);
    for (int q = tid; q < nd; q += blockDim.x) {
      if (done[q]) continue;
      cd* rq = dr + (int64_t)q * W;
      cd rp = rq[pi];
      for (int i = 0; i < W; ++i)
        if (i != pi) rq[i] = cfma(mu[i], rp, rq[i]);
      rq[pi] = cmul(rp, csub(tw_at(wN, did[q] / NS), sb));
    }
    // B* <- B* E
    int lmax = 0;
    for (int i = 0; i < W; ++i) lmax = max(lmax, blen[i * W + pi]);
    for (int idx = tid; idx < W * (lmax + 1); idx += blockDim.x) {
      int i = idx / (lmax + 1), t = idx % (lmax + 1);
      scr[(int64_t)i * B.cap + t] = t < blen[i * W + pi] ? bc[(int64_t)(i * W + pi) * B.cap + t] : mkc(0.0, 0.0);
    }
    __syncthreads();
    for (int idx = tid; idx < W * (lmax + 1); idx += blockDim.x) {
      int i = idx / (lmax + 1), t = idx % (lmax + 1);
      int lo = blen[i * W + pi];
      if (lo == 0 || t > lo || t >= B.cap) continue;
      cd o = t < lo ? scr[(int64_t)i * B.cap + t] : mkc(0.0, 0.0);
      cd prev = t >= 1 ? scr[(int64_t)i * B.cap + t - 1] : mkc(0.0, 0.0);
      bc[(int64_t)(i * W + pi) * B.cap + t] = csub(prev, cmul(sb, o));
      if (t < lo)
        for (int j = 0; j < W; ++j) {
          if (j == pi) continue;
          cd* dst = bc + (int64_t)(i * W + j) * B.cap + t;
          cd cur = t < blen[i * W + j] ? *dst : mkc(0.0, 0.0);
          *dst = cfma(mu[j], o, cur);
        }
    }
    __syncthreads();
    if (tid < W) {
      int i = tid, lo = blen[i * W + pi];
      if (lo > 0) {
        for (int j = 0; j < W; ++j)
          if (j != pi && blen[i * W + j] < lo) blen[i * W + j] = lo;
        blen[i * W + pi] = min(lo + 1, (int)B.cap);
        if (lo + 1 > B.cap) set_status(status, ST_DEGREE);
      }
    }
    if (tid == 0) dl[pi] += 1;
    __syncthreads();
  }
  if (tid < WW) B.lp(pb)[tid] = blen[tid];
  if (tid < W) {
    dlt[tid] = dl[tid];
    B.mp(pb)[tid] = (unsigned long long)__double_as_longlong(0.5);  // scale 1
  }
}

template <int W, int NS>
static int launch_difficult_t(Plan& P) {
  const int slots = std::min(P.opts.max_difficult, 64);
  k_diff_values<W, NS><<<dim3(W * W, slots, P.nb), 256, 0, P.stream>>>(P.buf[0][0], P.wN, P.N, P.ndiff, P.diff,
                                                                       P.opts.max_difficult, P.dvals);
  k_diff_rows<W, NS><<<dim3((unsigned)std::min(64, (W * P.opts.max_difficult + 255) / 256), P.nb), 256, 0,
                       P.stream>>>(P.Phi, P.N, P.ndiff, P.diff, P.opts.max_difficult, P.dvals, P.diffr);
  k_diff_serial<W, NS><<<P.nb, 1024, 0, P.stream>>>(P.buf[0][0], P.wN, P.ndiff, P.diff, P.opts.max_difficult,
                                                    P.diffr, P.delta, P.status, P.dscr, P.dscr_stride);
  return cudaGetLastError() == cudaSuccess ? 3 : TIKH_ECUDA;
}

int launch_difficult(Plan& P) { return P.w == 7 ? launch_difficult_t<7, 3>(P) : launch_difficult_t<5, 2>(P); }

}  // namespace tikh
