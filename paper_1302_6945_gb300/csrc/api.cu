// api.cu -- planning, workspace and the C-ABI entry points of include/tikh.h.
//
// Planning follows Algorithm 2 (OptExtend, Sec. 6.2) for two condition sets with paired
// interleaving: halve M while 2M > N_lim, make M even, and round it up to a 7-smooth value so every
// transform length factors into radices 2, 3, 4, 5, 7, 8; N = 2^p M, k = N - (m+n-1).  The DFS of
// Algorithm 1 is laid out once on the host as a list of steps; product transform lengths come from
// a water-filling model of the tau-degrees (every condition raises the lowest column) plus slack,
// and the device checks the real degrees against them (TIKH_EDEGREE triggers a re-plan and re-run).
// A plan serves up to opts.batch problems of one shape per call: every step is one launch for all.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

using namespace tikh;

struct tikh_plan_s {
  Plan P;
};

namespace {

bool is_5smooth(int64_t v) {
  if (v < 1) return false;
  for (int q : {2, 3, 5})
    while (v % q == 0) v /= q;
  return v == 1;
}
bool is_7smooth(int64_t v) {
  if (v < 1) return false;
  for (int q : {2, 3, 5, 7})
    while (v % q == 0) v /= q;
  return v == 1;
}
int64_t smooth_at_least(int64_t v) {
  if (v < 2) v = 2;
  while (!is_5smooth(v)) ++v;
  return v;
}

// the automatic direct/FFT thresholds for `items` items per launch (a single item: the latency-bound forms)
void auto_thresholds(int64_t items, int prec, int& prod, int& eval) {
  if (items == 1 || prec != TIKH_PREC_FP64) { prod = 360; eval = 80; return; }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const bool full = items >= sms;
  prod = full ? FULL_BATCH_PROD_DIRECT_MAX : BATCH_PROD_DIRECT_MAX;
  eval = full ? FULL_BATCH_EVAL_DIRECT_MAX : BATCH_EVAL_DIRECT_MAX;
}

void* dalloc(Plan& P, size_t bytes, int& err) {
  if (err) return nullptr;
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    err = TIKH_ENOMEM;
    return nullptr;
  }
  P.allocs.push_back(p);
  P.bytes += (int64_t)bytes;
  return p;
}

cd* twiddle(Plan& P, int64_t L, int& err) {
  auto it = P.twiddle_of_len.find(L);
  if (it != P.twiddle_of_len.end()) return it->second;
  cd* t = (cd*)dalloc(P, sizeof(cd) * (size_t)L, err);
  if (err) return nullptr;
  if (launch_twiddle(t, L, P.stream) < 0) { err = TIKH_ECUDA; return nullptr; }
  P.twiddle_of_len[L] = t;
  return t;
}

cf* twiddle32(Plan& P, int64_t L, int& err) {
  auto it = P.twiddle32_of_len.find(L);
  if (it != P.twiddle32_of_len.end()) return it->second;
  cd* src = twiddle(P, L, err);
  cf* t = (cf*)dalloc(P, sizeof(cf) * (size_t)L, err);
  if (err) return nullptr;
  if (launch_to_cf(src, t, L, P.stream) < 0) { err = TIKH_ECUDA; return nullptr; }
  P.twiddle32_of_len[L] = t;
  return t;
}

int fft_index(Plan& P, int64_t L, int& err) {
  auto it = P.fft_of_len.find(L);
  if (it != P.fft_of_len.end()) return it->second;
  FftPlan f;
  f.L = L;
  f.tile = P.opts.fft_tile > 0 ? P.opts.fft_tile : 256;
  const int rmax = P.opts.fft_radix > 0 ? P.opts.fft_radix : 8;
  if (L <= FFT_TILE_MAX) {
    if (!fft_factor((int)L, f.d1, rmax)) { err = TIKH_EINVAL; return -1; }
    f.d1.tw = twiddle(P, L, err);
  } else {
    int64_t L1, L2;
    if (!fft_split(L, L1, L2)) { err = TIKH_EINVAL; return -1; }
    f.four = true;
    f.L1 = L1;
    f.L2 = L2;
    fft_factor((int)L1, f.d1, rmax);
    fft_factor((int)L2, f.d2, rmax);
    f.d1.tw = twiddle(P, L1, err);
    f.d2.tw = twiddle(P, L2, err);
    f.twL = twiddle(P, L, err);
  }
  if (P.stage32 && !err) {  // complex64 tables for the FP32 stages
    if (!f.four) {
      f.d1.tw32 = twiddle32(P, L, err);
    } else {
      f.d1.tw32 = twiddle32(P, f.L1, err);
      f.d2.tw32 = twiddle32(P, f.L2, err);
      f.twL32 = twiddle32(P, L, err);
    }
  }
  if (err) return -1;
  P.ffts.push_back(f);
  P.fft_of_len[L] = (int)P.ffts.size() - 1;
  return (int)P.ffts.size() - 1;
}

// same bound as the device: tau-degree bound for pivoted columns, accumulation bound otherwise
int entry_bound_host(int W, const int* din, const int* dout, int i, int j) {
  int amax = 0;
  bool have = false;
  for (int c = 0; c < W; ++c)
    if (dout[c] > din[c]) { amax = have ? std::max(amax, dout[c]) : dout[c]; have = true; }
  if (dout[j] > din[j]) return dout[j] - din[i];
  int acc = have ? amax - din[i] : -1;
  if (i == j && acc < 0) acc = 0;
  return std::min(acc, dout[j] - din[i]);
}

void waterfill(int W, int* d, int64_t C) {
  for (int64_t c = 0; c < C; ++c) {
    int j = 0;
    for (int i = 1; i < W; ++i)
      if (d[i] < d[j]) j = i;
    d[j] += 1;
  }
}

// The DFS of Algorithm 1 for one shape: leaves, evaluations and products in execution order, with the
// product transform length predicted from the shape's tau-degrees (water-filling) plus slack.
void build_steps(Plan& P, std::vector<Step>& out, int depth, int64_t a, int64_t s, int64_t L, int side, int* sd,
                 uint64_t& pending, int64_t slack) {
  const int W = P.w, NS = P.ns;
  if (depth == P.p) {
    // the leaf saves its delta_in for its own depth too: the product of its parent reads the right leaf's
    Step st{STEP_LEAF, depth, side, a, s, L, -1, 0, pending | (1ULL << depth)};
    pending = 0;
    waterfill(W, sd, 2 * NS * L);
    out.push_back(st);
    return;
  }
  int din[WMAX];
  memcpy(din, sd, sizeof(int) * W);
  pending |= (1ULL << depth);
  build_steps(P, out, depth + 1, a, 2 * s, L / 2, 0, sd, pending, slack);
  int dmid[WMAX];
  memcpy(dmid, sd, sizeof(int) * W);
  unsigned sl = 0u, sr = 0u;
  for (int j = 0; j < W; ++j) sl |= (dmid[j] > din[j] ? 1u : 0u) << j;
  Step ev{STEP_EVAL, depth, side, a, s, L, -1, 0, 0};
  ev.sl = sl;
  out.push_back(ev);
  build_steps(P, out, depth + 1, a + s, 2 * s, L / 2, 1, sd, pending, slack);
  for (int j = 0; j < W; ++j) sr |= (sd[j] > dmid[j] ? 1u : 0u) << j;
  int D = -1;
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j) D = std::max(D, entry_bound_host(W, din, sd, i, j));
  // the product of the bases of 2 NS L conditions has degree <= 2 NS L whatever the tau-degree bound and
  // the slack say, and each child's stored entries are at most NS L + 1 long (they are trimmed to the
  // same kind of bound), which the transform must hold
  int64_t Pn = smooth_at_least(
      std::max<int64_t>(NS * L + 1, std::min<int64_t>((int64_t)D + 1 + slack, 2 * NS * L + 1)));
  Step pr{STEP_PROD, depth, side, a, s, L, -1, Pn, 0};
  pr.sl = sl;
  pr.sr = sr;
  out.push_back(pr);
}

// Algorithmic FLOPs of one item's core solve by kind (leaf, evaluation, product, other), the part the FFT
// stages run in FP32 kept apart: a length-L complex FFT counts 5 L log2 L, a complex multiply-add 8.
// W = basis size (5, or 7 for the general problem), NS = condition sets per node (2, or 3).
//  leaf of K = 2 NS L conditions: (W/5)(30 K^2 + 90 K) for the pivot chain (a sum over steps of 60 per
//    remaining condition and 90 per step at W = 5, both proportional to the row length W) plus
//    (W^2/25) 20 K^2 for the basis rebuild (W^2 entries); 50 K^2 + 90 K at W = 5;
//  evaluation at Lr = L/2 nodes per coset: direct, 2 Lr nodes x W^2 entries x len Horner steps; FFT, the
//    twist-fold (2 |S_L| W x len) and 2 |S_L| W transforms of Lr (the identity rows of B_L, outside the
//    columns S_L the left child pivots, are not transformed); both plus the update, 2 Lr nodes x NS rows x
//    W^2 CMACs; len = NS L / W + 1 is the mean entry length of the left child (its NS L conditions raise
//    each of the W columns by NS L / W);
//  product of length P: direct, W^2 outputs x W convolutions of len x len; FFT, one transform of P per
//    operand entry outside the identity rows ((|S_L| + |S_R|) W) and per output entry in the rows S_L u S_R,
//    and W pointwise CMACs per output entry and bin; on the right spine (no deferred condition assumed)
//    only column j*: |S_L| W + |S_R| operand and |S| output transforms, and at the root only rows 0 and
//    W - 1 of B_L and those two rows of the output;  S_L, S_R from the water-filling prediction;
//  other: the length-N transforms of the extension (one more for L or G), right-hand side and conditions.
void model_flops(Plan& P) {
  auto fft = [](double L) { return L > 1 ? 5.0 * L * std::log2(L) : 0.0; };
  const double W = P.w, WW = W * W, NS = P.ns;
  for (int k = 0; k < 4; ++k) P.last.model_flops[k] = P.last.model_flops_fp32[k] = 0.0;
  for (const Step& st : P.sched) {
    const double L = (double)st.L, Lr = L / 2, len = NS * L / W + 1.0;
    if (st.kind == STEP_LEAF) {
      const double K = 2 * NS * L;
      P.last.model_flops[0] += (W / 5) * (30 * K * K + 90 * K) + (WW / 25) * 20 * K * K;
    } else if (st.kind == STEP_EVAL) {
      const double upd = 2 * Lr * NS * WW * 8;
      const double nsl = __builtin_popcount(st.sl);
      if (st.L / 2 <= P.eval_direct_max) {
        P.last.model_flops[1] += 2 * Lr * WW * len * 8 + upd;
      } else {
        const double f = 2 * nsl * W * len * 8 + 2 * nsl * W * fft(Lr) + upd;
        P.last.model_flops[1] += f;
        if (P.stage32) P.last.model_flops_fp32[1] += f;
      }
    } else {
      const double Pl = (double)st.P;
      if (st.P <= P.prod_direct_max) {
        P.last.model_flops[2] += WW * W * len * len * 8;
      } else {
        const int mode = st.depth == 0 ? 2 : (st.a == st.s - 2 ? 1 : 0);  // the root, the right spine, other
        const unsigned su = st.sl | st.sr;
        const double nsl = __builtin_popcount(st.sl), nsr = __builtin_popcount(st.sr), nsu = __builtin_popcount(su);
        const double ends = (double)((su & 1u) != 0) + (double)(((su >> (P.w - 1)) & 1u) != 0);  // rows 0, W - 1
        const double endsl = (double)((st.sl & 1u) != 0) + (double)(((st.sl >> (P.w - 1)) & 1u) != 0);
        double operands, outputs;
        if (mode == 0) { operands = (nsl + nsr) * W; outputs = nsu * W; }
        else if (mode == 1) { operands = nsl * W + nsr; outputs = nsu; }
        else { operands = endsl * W + nsr; outputs = ends; }
        const double f = (operands + outputs) * fft(Pl) + outputs * W * Pl * 8;
        P.last.model_flops[2] += f;
        if (P.stage32) P.last.model_flops_fp32[2] += f;
      }
    }
  }
  P.last.model_flops[3] = (P.gram || P.general ? 5 : 4) * fft((double)P.N);
}

// (re)build the schedule for every shape the plan serves (the step list is the same for all of them --
// it depends on N, p, M only -- and each product takes the largest length any shape predicts), then
// the FFT plans, the product scratch and the basis buffers
int make_schedule(Plan& P) {
  int err = 0;
  const size_t nb = (size_t)P.batch_max;
  P.sched.clear();
  for (const Shape& sh : P.shapes) {
    std::vector<Step> st;
    int sd[WMAX] = {-(int)(sh.cn - 1), -(int)(sh.cm - 1), -(int)(sh.cm + sh.k - 2), -(int)(sh.cn + sh.k - 2), 0, 0, 0};
    if (P.general) {  // tau = [n-1, m-1, pl-1, N-n-1, N-m-1, N-pl-1, 0]
      const int64_t t[WMAX] = {sh.cn - 1, sh.cm - 1, sh.pl - 1, P.N - sh.cn - 1, P.N - sh.cm - 1, P.N - sh.pl - 1, 0};
      for (int i = 0; i < WMAX; ++i) sd[i] = -(int)t[i];
    }
    uint64_t pending = 0;
    const int64_t slack = (int64_t)P.slack_mult * (std::max(sh.k, sh.kl) + P.ns * P.M + 4);
    build_steps(P, st, 0, 0, 2, P.N / 2, 0, sd, pending, slack);
    if (P.sched.empty()) {
      P.sched = st;
    } else {
      for (size_t i = 0; i < st.size(); ++i) P.sched[i].P = std::max(P.sched[i].P, st[i].P);
    }
  }
  int64_t oldP = P.Pmax;
  for (Step& st : P.sched) {
    if (st.kind == STEP_PROD) P.Pmax = std::max(P.Pmax, st.P);
    if (st.kind == STEP_EVAL) {
      st.fft = fft_index(P, st.L / 2, err);
      P.Lrmax = std::max(P.Lrmax, st.L / 2);
    } else if (st.kind == STEP_PROD) {
      st.fft = fft_index(P, st.P, err);
    }
  }
  if (err) return err;
  model_flops(P);
  const size_t WW = (size_t)P.w * P.w;
  if (P.Pmax > oldP || !P.FA) {
    size_t nww = WW * (size_t)std::max<int64_t>(P.Pmax, 1) * nb;
    P.FA = (cd*)dalloc(P, sizeof(cd) * nww, err);
    P.FB = (cd*)dalloc(P, sizeof(cd) * nww, err);
    P.FC = (cd*)dalloc(P, sizeof(cd) * nww, err);
    P.ptmp = (cd*)dalloc(P, sizeof(cd) * 2 * nww, err);
  }
  // basis capacity per depth: a product's entries are at most P long (P exceeds every entry degree
  // bound of the node, which can exceed the node's condition count by the spread of delta_in);
  // leaves hold at most K + 1 = NS M + 1 coefficients; the root also absorbs the difficult points
  int64_t need[MAX_DEPTH] = {0};
  need[P.p] = P.ns * P.M + 1;
  for (const Step& st : P.sched)
    if (st.kind == STEP_PROD) need[st.depth] = std::max(need[st.depth], st.P);
  need[0] += std::min(P.opts.max_difficult, 4096) + 2;
  for (int d = 0; d <= P.p && !err; ++d)
    for (int side = 0; side < (d == 0 ? 1 : 2); ++side) {
      BasisBuf& B = P.buf[d][side];
      if (B.cap >= need[d]) continue;
      B.cap = need[d];
      B.ww = (int)WW;
      B.c = (cd*)dalloc(P, sizeof(cd) * WW * (size_t)B.cap * nb, err);
      if (!B.len) B.len = (int*)dalloc(P, sizeof(int) * 64 * nb, err);
      if (!B.colmax) B.colmax = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * 8 * nb, err);
      if (d == 0) {
        P.dscr_stride = P.w * B.cap + P.opts.max_difficult;
        P.dscr = (cd*)dalloc(P, sizeof(cd) * (size_t)P.dscr_stride * nb, err);
      }
    }
  return err;
}

int status_to_code(int st) {
  if (st & ST_WAIT) return TIKH_ETIMEOUT;
  if (st & ST_INPUT) return TIKH_ENUMERIC;
  if (st & ST_DIFFICULT) return TIKH_EDIFFICULT;
  if (st & ST_DEGREE) return TIKH_EDEGREE;
  if (st & ST_NUMERIC) return TIKH_ENUMERIC;
  return TIKH_OK;
}

// profiling: an event pair around one launch group, kind 0..3 (leaf, evaluation, product, other)
struct ProfScope {
  Plan& P;
  cudaEvent_t e1 = nullptr;
  ProfScope(Plan& p, int kind) : P(p) {
    const bool on = (P.prof_leaf & 2) || (kind == 0 && (P.prof_leaf & 1));
    if (!on) return;
    while (P.ev_pool.size() < P.ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      P.ev_pool.push_back(e);
    }
    if (P.ev_kind.size() < P.ev_pool.size() / 2) P.ev_kind.resize(P.ev_pool.size() / 2);
    cudaEventRecord(P.ev_pool[P.ev_used], P.stream);
    e1 = P.ev_pool[P.ev_used + 1];
    P.ev_kind[P.ev_used / 2] = (signed char)kind;
    P.ev_used += 2;
  }
  ~ProfScope() {
    if (e1) cudaEventRecord(e1, P.stream);
  }
};

// one superfast solve of every problem's core system with right-hand side y, solution into out
int enqueue_core(Plan& P, const cd* y, cd* out, int64_t& nl) {
  int r;
  {
    ProfScope ps(P, 3);
    if ((r = launch_conditions(P, y)) < 0) return r;
  }
  nl += r;
  for (const Step& st : P.sched) {
    if (st.kind == STEP_LEAF) {
      ProfScope ps(P, 0);
      r = launch_leaf(P, st);
    } else if (st.kind == STEP_EVAL) {
      ProfScope ps(P, 1);
      r = launch_eval(P, st);
    } else {
      ProfScope ps(P, 2);
      r = launch_prod(P, st);
    }
    if (r < 0) return r;
    nl += r;
  }
  {
    ProfScope ps(P, 3);
    if ((r = launch_difficult(P)) < 0) return r;
    nl += r;
    if ((r = launch_extract(P, out)) < 0) return r;
  }
  nl += r;
  return TIKH_OK;
}

// core solve of A v = y (y in P.ybuf) into P.xcore, then opts.refine_steps corrections
int enqueue_core_refined(Plan& P, int64_t& nl) {
  int r;
  if ((r = enqueue_core(P, P.ybuf, P.xcore, nl)) < 0) return r;
  // iterative refinement on the core system: v <- v + A^{-1}(y - A v)
  for (int it = 0; it < P.opts.refine_steps; ++it) {
    {
      ProfScope ps(P, 3);
      if ((r = launch_residual(P, P.ybuf, P.xcore, P.rbuf)) < 0) return r;
    }
    nl += r;
    if ((r = enqueue_core(P, P.rbuf, P.dx, nl)) < 0) return r;
    {
      ProfScope ps(P, 3);
      if ((r = launch_axpy(P, P.xcore, P.dx)) < 0) return r;
    }
    nl += r;
  }
  if (P.opts.refine_steps > 0) {  // residual of the refined solution, reported in the stats
    ProfScope ps(P, 3);
    if ((r = launch_residual(P, P.ybuf, P.xcore, P.rbuf)) < 0) return r;
    nl += r;
  }
  return TIKH_OK;
}

// items and lambdas of a call into the device tables at offset `off` (outside any graph: a replay reads
// whatever the tables hold)
int stage_items(Plan& P, const ItemDev* items, const double* lams, int nb, int64_t off) {
  if (nb < 1 || off + nb > P.item_cap) return TIKH_EINVAL;
  if (cudaMemcpyAsync(P.items_base + off, items, sizeof(ItemDev) * (size_t)nb, cudaMemcpyHostToDevice, P.stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(P.lam_base + off, lams, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, P.stream) !=
          cudaSuccess)
    return TIKH_ECUDA;
  return TIKH_OK;
}

int enqueue_prologue(Plan& P, int rhs_is_y, int nb, int64_t& nl) {
  int r;
  if (nb < 1 || nb > P.batch_max) return TIKH_EINVAL;
  P.nb = nb;
  if (!P.keep_status && cudaMemsetAsync(P.status, 0, sizeof(int), P.stream) != cudaSuccess) return TIKH_ECUDA;
  ProfScope ps(P, 3);
  if ((r = launch_spectrum(P, rhs_is_y)) < 0) return r;
  nl += r;
  // for m < n the core problem (T T^H + lam I) v = b takes b itself as its right-hand side
  if ((r = launch_rhs(P, P.dual ? 1 : rhs_is_y)) < 0) return r;
  nl += r;
  return TIKH_OK;
}

// the whole solve of the nb staged items (P.items, P.lam) on the plan's stream
int enqueue_solve(Plan& P, int rhs_is_y, int nb) {
  int64_t nl = 0;
  int r;
  if ((r = enqueue_prologue(P, rhs_is_y, nb, nl)) < 0) return r;
  if ((r = enqueue_core_refined(P, nl)) < 0) return r;
  {
    ProfScope ps(P, 3);
    if ((r = launch_output(P, P.xcore)) < 0) return r;
  }
  nl += r;
  P.launches = nl;
  return TIKH_OK;
}

void drop_graph(Plan& P) {
  if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
  P.graph_exec = nullptr;
  P.graph_nb = 0;
}

// the solve as a CUDA graph: the item and lambda tables are staged outside the graph; the rest (status
// reset, transform, every node of the recursion, refinement, output) is captured once per item count
// and replayed -- it reads the arrays and sizes of each call from the tables
int enqueue_solve_graph(Plan& P, int rhs_is_y, int nb) {
  if (nb < 1 || nb > P.batch_max) return TIKH_EINVAL;
  if (!P.graph_exec || P.graph_nb != nb || P.graph_rhs_is_y != rhs_is_y) {
    drop_graph(P);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();  // e.g. the legacy default stream, which cannot be captured
      P.opts.graph = 0;
      return enqueue_solve(P, rhs_is_y, nb);
    }
    int rc = enqueue_solve(P, rhs_is_y, nb);
    cudaError_t ce = cudaStreamEndCapture(P.stream, &g);
    if (rc || ce != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      P.opts.graph = 0;  // capture not possible here: plain stream launches from now on
      return rc ? rc : enqueue_solve(P, rhs_is_y, nb);
    }
    ce = cudaGraphInstantiate(&P.graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      P.graph_exec = nullptr;
      P.opts.graph = 0;
      return enqueue_solve(P, rhs_is_y, nb);
    }
    P.graph_nb = nb;
    P.graph_rhs_is_y = rhs_is_y;
  }
  P.nb = nb;
  return cudaGraphLaunch(P.graph_exec, P.stream) == cudaSuccess ? TIKH_OK : TIKH_ECUDA;
}

int enqueue_any(Plan& P, int rhs_is_y, int nb) {
  P.last.graph = 0;
  if (P.opts.graph && !P.prof_leaf) {
    int rc = enqueue_solve_graph(P, rhs_is_y, nb);
    P.last.graph = P.graph_exec && P.opts.graph ? 1 : 0;
    return rc;
  }
  return enqueue_solve(P, rhs_is_y, nb);
}

int sync_status(Plan& P) {
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) { cudaGetLastError(); return TIKH_ECUDA; }
  int st = 0;
  if (cudaMemcpy(&st, P.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TIKH_ECUDA;
  std::vector<int> nd(4 * (size_t)P.nb), dl(DSTR * (size_t)P.nb);
  cudaMemcpy(nd.data(), P.ndiff, sizeof(int) * nd.size(), cudaMemcpyDeviceToHost);
  cudaMemcpy(dl.data(), P.delta, sizeof(int) * dl.size(), cudaMemcpyDeviceToHost);
  int64_t total = 0;
  for (int b = 0; b < P.nb; ++b) total += nd[4 * b];
  P.last.n_difficult = total;
  for (int j = 0; j < 7; ++j) P.last.delta[j] = j < P.w ? dl[j] : 0;
  P.last.jstar = -1;
  for (int j = 0; j < P.w; ++j)
    if (dl[j] == 0) P.last.jstar = j;
  P.last.kernel_launches = P.launches;
  P.last.refine_steps = P.opts.refine_steps;
  P.last.batch = P.nb;
  P.last.rel_residual = -1.0;
  P.last.last_correction = -1.0;
  if (P.opts.refine_steps > 0) {  // largest relative residual of the batch
    std::vector<double> nr(4 * (size_t)P.nb);
    cudaMemcpy(nr.data(), P.norms, sizeof(double) * nr.size(), cudaMemcpyDeviceToHost);
    double worst = 0.0, corr = 0.0;
    for (int b = 0; b < P.nb; ++b) {
      double v = nr[4 * b + 1] > 0.0 ? sqrt(nr[4 * b] / nr[4 * b + 1]) : sqrt(nr[4 * b]);
      worst = std::max(worst, v);
      corr = std::max(corr, nr[4 * b + 3] > 0.0 ? sqrt(nr[4 * b + 2] / nr[4 * b + 3]) : 0.0);
    }
    P.last.rel_residual = worst;
    P.last.last_correction = corr;
  }
  if (P.prof_leaf) {  // durations of the event pairs recorded since the last sync, accumulated until
                      // tikh_set_profiling re-arms it
    for (size_t i = 0; i + 1 < P.ev_used; i += 2) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, P.ev_pool[i], P.ev_pool[i + 1]) != cudaSuccess) continue;
      const int kind = P.ev_kind[i / 2];
      if (kind == 0) {
        P.last.prof_leaf_ms += t;
        P.last.prof_leaf_launches += 1;
      }
      if (P.prof_leaf & 2) {
        P.last.prof_kind_ms[kind] += t;
        P.last.prof_kind_count[kind] += 1;
      }
    }
    P.ev_used = 0;
  }
  int zero = 0;
  cudaMemcpy(P.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
  int code = status_to_code(st);
  // the refinement's tolerance (opts.refine_tol > 0): a residual still above it is reported
  if (code == TIKH_OK && P.opts.refine_tol > 0.0 && P.opts.refine_steps > 0 &&
      !(P.last.rel_residual <= P.opts.refine_tol))
    code = TIKH_ENOTCONVERGED;
  return code;
}

// stage the items, solve, optionally copy x (device x_dev) back to the host, synchronise; re-plan with
// more degree slack and re-run after TIKH_EDEGREE
int solve_with_retry(Plan& P, const std::vector<ItemDev>& items, const double* lams, int rhs_is_y, void* x_host,
                     const void* x_dev, size_t xbytes) {
  P.last.retries = 0;
  const int nb = (int)items.size();
  P.items = P.items_base;
  P.lam = P.lam_base;
  P.keep_status = false;
  for (int attempt = 0;; ++attempt) {
    int rc = stage_items(P, items.data(), lams, nb, 0);
    if (rc) return rc;
    if ((rc = enqueue_any(P, rhs_is_y, nb))) return rc;
    if (x_host && cudaMemcpyAsync(x_host, x_dev, xbytes, cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
      return TIKH_ECUDA;
    rc = sync_status(P);
    if (rc != TIKH_EDEGREE || attempt >= 3) return rc;
    P.slack_mult *= 16;
    P.last.retries = attempt + 1;
    drop_graph(P);
    if ((rc = make_schedule(P))) return rc;
  }
}

bool valid_lambda(double lam) { return lam > 0.0 && lam < 1e300; }

ItemDev make_item(const Shape& sh, const void* col, const void* row, const void* rhs, void* x) {
  ItemDev it;
  memset(&it, 0, sizeof(it));  // gram = null: the l2 problem
  it.col = col;
  it.row = row;
  it.rhs = rhs;
  it.x = x;
  it.m = sh.m;
  it.n = sh.n;
  it.cm = sh.cm;
  it.cn = sh.cn;
  it.k = sh.k;
  it.dual = sh.dual;
  return it;
}

std::vector<ItemDev> single(const Plan& P, const void* col, const void* row, const void* rhs, void* x) {
  return std::vector<ItemDev>(1, make_item(P.shapes[0], col, row, rhs, x));
}

// Algorithm 2 (reading: two condition sets, paired interleaving; M even, 7-smooth) for the core problem
// cm x cn: halve M while 2M > N_lim, round up to even and 7-smooth; N = 2^p M, k = N - (cm + cn - 1)
// Algorithm 2 for ns condition sets per node over a circulant of at least Nt points: halve M while
// ns M > N_lim; a leaf then holds ns M conditions, at most kmax (64 for the 5 x 5 basis, 42 for 7 x 7)
bool alg2_sets(int64_t Nt, int ns, int kmax, const tikh_opts& o, int64_t& N, int64_t& M, int& p) {
  int64_t Mv = Nt;
  int pv = 0;
  while (ns * Mv > o.n_lim) { ++pv; Mv = (Mv + 1) / 2; }
  if (Mv % 2) ++Mv;
  if (Mv < o.m_min) Mv = o.m_min + (o.m_min % 2);
  while (!is_7smooth(Mv)) Mv += 2;
  M = Mv;
  p = pv;
  N = Mv << pv;
  return !(pv >= MAX_DEPTH - 1 || ns * Mv > kmax || N > (int64_t)1 << 31);
}

bool alg2(int64_t cm, int64_t cn, const tikh_opts& o, int64_t& N, int64_t& M, int& p) {
  return alg2_sets(cm + cn - 1, 2, 64, o, N, M, p);
}

bool valid_prec(int prec) {
  return prec == TIKH_PREC_FP64 || prec == TIKH_PREC_FP32_REFINE || prec == TIKH_PREC_FP32;
}

bool valid_opts(const tikh_opts& o) {
  return !(o.n_lim < 4 || o.n_lim > 64 || o.m_min < 0 || o.m_min > 32 || (o.fill != 0 && o.fill != 1) ||
           !(o.eps_diff >= 0.0) || o.max_difficult < 1 || o.max_difficult > (1 << 20) || o.refine_steps < 0 ||
           o.refine_steps > 8 || o.batch < 1 || o.batch > 65535 || (o.graph != 0 && o.graph != 1) ||
           o.prod_direct_max < 0 || o.prod_direct_max > 4096 || o.eval_direct_max < 0 || o.eval_direct_max > 4096 ||
           o.wait_polls < 0 || o.wait_polls > (1 << 30) || !(o.refine_tol >= 0.0) ||
           (o.fft_radix != 0 && o.fft_radix != 4 && o.fft_radix != 8) || o.fft_tile < 0 || o.fft_tile > 4096 ||
           (o.fft_tile & (o.fft_tile - 1)) != 0);
}

Shape core_shape(int64_t m, int64_t n, int64_t N) {
  Shape sh;
  sh.m = m;
  sh.n = n;
  sh.dual = m < n ? 1 : 0;
  sh.cm = sh.dual ? n : m;
  sh.cn = sh.dual ? m : n;
  sh.k = N - (sh.cm + sh.cn - 1);
  return sh;
}

void set_profiling(Plan& P, int flags) {
  P.prof_leaf = flags & 3;
  P.ev_used = 0;
  P.last.prof_leaf_ms = 0.0;
  P.last.prof_leaf_launches = 0;
  for (int k = 0; k < 4; ++k) {
    P.last.prof_kind_ms[k] = 0.0;
    P.last.prof_kind_count[k] = 0;
  }
}

void free_plan(Plan& P) {
  cudaStreamSynchronize(P.stream);
  drop_graph(P);
  for (cudaEvent_t e : P.ev_pool) cudaEventDestroy(e);
  P.ev_pool.clear();
  for (void* p : P.allocs) cudaFree(p);
  P.allocs.clear();
}

// Plan for problems of the given shapes (all sharing N, M, p and the dual flag), up to o.batch items per
// call: schedule, FFT plans, twiddles and every device buffer.  P.m, P.n, P.cm, P.cn are the largest
// over the shapes (buffer strides); P.k is that of the first shape.
int plan_setup(Plan& P, const std::vector<Shape>& shapes, int64_t N, int64_t M, int p, int dtype, int prec,
               const tikh_opts& o, cudaStream_t stream, int64_t item_cap) {
  P.dtype = dtype;
  P.prec = prec;
  P.stage32 = prec != TIKH_PREC_FP64;
  P.opts = o;
  // the FP32 pattern refines in FP64: two corrections unless the caller asks for a number
  if (prec == TIKH_PREC_FP32_REFINE && P.opts.refine_steps == 0) P.opts.refine_steps = 2;
  P.batch_max = o.batch;
  // direct vs FFT forms of steps 2 and 4: a single problem is latency-bound at small nodes (direct forms
  // spread over more SMs with short chains); a batch is FP64-throughput-bound, where the O(P^2) direct
  // product loses to the O(P log P) FFT product at much smaller P (measured on GB300)
  // product; with FP32 stages the small nodes stay on the FP64 direct forms whatever the batch: the FP32 FFT
  // forms at the many small nodes dominate the error (measured: 1e-4 .. divergence in batches with the batch
  // thresholds, 3e-5 per solve with these)
  int auto_prod, auto_eval;
  auto_thresholds(o.batch, prec, auto_prod, auto_eval);
  P.prod_direct_max = o.prod_direct_max > 0 ? o.prod_direct_max : auto_prod;
  P.eval_direct_max = o.eval_direct_max > 0 ? o.eval_direct_max : auto_eval;
  P.wait_polls = o.wait_polls > 0 ? o.wait_polls : (1 << 24);
  P.stream = stream;
  P.shapes = shapes;
  P.dual = shapes[0].dual;
  P.N = N;
  P.M = M;
  P.p = p;
  P.k = shapes[0].k;
  P.m = P.n = P.cm = P.cn = P.pl = 0;
  for (const Shape& sh : shapes) {
    P.m = std::max(P.m, sh.m);
    P.n = std::max(P.n, sh.n);
    P.cm = std::max(P.cm, sh.cm);
    P.cn = std::max(P.cn, sh.cn);
    P.pl = std::max(P.pl, sh.pl);
  }
  const size_t rw = (size_t)P.ns * P.w;  // residual entries per node
  int err = 0;
  const size_t nb = (size_t)P.batch_max;
  if (fft_index(P, P.N, err) < 0 && !err) err = TIKH_EINVAL;
  P.wN = err ? nullptr : P.twiddle_of_len[P.N];
  if (P.stage32 && !err) P.wN32 = twiddle32(P, P.N, err);
  P.specT = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
  P.work = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
  P.work2 = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
  P.ftmpN = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
  P.R = (cd*)dalloc(P, sizeof(cd) * rw * (size_t)N * nb, err);
  P.Phi = (cd*)dalloc(P, sizeof(cd) * rw * (size_t)N * nb, err);
  P.delta = (int*)dalloc(P, sizeof(int) * DSTR * nb, err);
  P.dstack = (int*)dalloc(P, sizeof(int) * DSTR * MAX_DEPTH * nb, err);
  P.status = (int*)dalloc(P, sizeof(int) * 4, err);
  P.ndiff = (int*)dalloc(P, sizeof(int) * 4 * nb, err);
  P.bad = (int*)dalloc(P, sizeof(int) * nb, err);
  P.diff = (int64_t*)dalloc(P, sizeof(int64_t) * (size_t)o.max_difficult * nb, err);
  P.diffr = (cd*)dalloc(P, sizeof(cd) * P.w * (size_t)o.max_difficult * nb, err);
  P.dvals = (cd*)dalloc(P, sizeof(cd) * P.w * P.w * (size_t)o.max_difficult * nb, err);
  P.peak = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * nb, err);
  P.item_cap = std::max<int64_t>(item_cap, (int64_t)nb);
  P.items_base = (ItemDev*)dalloc(P, sizeof(ItemDev) * (size_t)P.item_cap, err);
  P.lam_base = (double*)dalloc(P, sizeof(double) * (size_t)P.item_cap, err);
  P.items = P.items_base;
  P.lam = P.lam_base;
  if (!err) err = make_schedule(P);
  if (!err) {
    size_t nl = 2 * (size_t)P.w * P.w * (size_t)std::max<int64_t>(P.Lrmax, 1) * nb;
    P.evalv = (cd*)dalloc(P, sizeof(cd) * nl, err);
    P.etmp = (cd*)dalloc(P, sizeof(cd) * nl, err);
    P.ybuf = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.rbuf = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.xcore = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.dx = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.norms = (double*)dalloc(P, sizeof(double) * 4 * nb, err);
    if (P.gram) {
      P.specG = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
      P.peakG = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * nb, err);
    }
    if (P.general) {
      P.specL = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
      P.peakL = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * nb, err);
    }
    if (P.gram || P.general) P.gX = (cd*)dalloc(P, sizeof(cd) * (size_t)N * nb, err);
  }
  if (!err && cudaStreamSynchronize(P.stream) != cudaSuccess) err = TIKH_ECUDA;
  if (err) {
    cudaGetLastError();
    free_plan(P);
    return err;
  }
  P.last.N = P.N;
  P.last.M = P.M;
  P.last.k = P.k;
  P.last.p = P.p;
  P.last.dual = P.dual;
  P.last.batch = 1;
  return TIKH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------------
// batch plans: problems of different shapes and a regularisation path, in one call
// ---------------------------------------------------------------------------------------------------

// One group of a batch plan: the problems whose core problems share N (and the m < n form), solved
// with one schedule in waves of up to W items (problem, lambda) on the group's own stream.
struct BatchGroup {
  Plan P;
  std::vector<int64_t> items;  // item ids prob * nlambda + l, in wave order
  int W = 0, waves = 0;
  cudaEvent_t done = nullptr;
  std::vector<cudaGraphExec_t> graphs;  // opts.graph: one captured graph per wave
};

struct tikh_batch_plan_s {
  int nprob = 0, nlambda = 0, dtype = 0;
  std::vector<int64_t> m, n;
  std::vector<int> group_of;  // problem -> group
  tikh_opts opts{};
  cudaStream_t stream = nullptr;
  std::vector<BatchGroup*> groups;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t launches = 0;
  int prof = 0;  // profiling flags of every group; groups then run one after another on `stream`
  tikh_batch_stats last{};
};

namespace {

void drop_wave_graphs(BatchGroup* g) {
  for (cudaGraphExec_t e : g->graphs)
    if (e) cudaGraphExecDestroy(e);
  g->graphs.clear();
}

void batch_free(tikh_batch_plan h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (BatchGroup* g : h->groups) {
    drop_wave_graphs(g);
    free_plan(g->P);
    if (g->done) cudaEventDestroy(g->done);
    if (g->P.stream) cudaStreamDestroy(g->P.stream);
    delete g;
  }
  if (h->fork) cudaEventDestroy(h->fork);
  delete h;
}

// every wave of every group, each group on its own stream forked from and joined to the plan's stream
int batch_enqueue(tikh_batch_plan h) {
  int64_t nl = 0;
  if (cudaEventRecord(h->fork, h->stream) != cudaSuccess) return TIKH_ECUDA;
  for (BatchGroup* g : h->groups) {
    Plan& P = g->P;
    if (h->prof) {  // profiled: every group in turn on the plan's stream
      cudaStream_t own = P.stream;
      P.stream = h->stream;
      int rc = TIKH_OK;
      for (int w = 0; w < g->waves && !rc; ++w) {
        const int64_t off = (int64_t)w * g->W;
        const int nb = (int)std::min<int64_t>(g->W, (int64_t)g->items.size() - off);
        P.items = P.items_base + off;
        P.lam = P.lam_base + off;
        P.keep_status = w > 0;
        rc = enqueue_solve(P, 0, nb);
        nl += P.launches;
      }
      P.stream = own;
      if (rc) return rc;
      continue;
    }
    if (cudaStreamWaitEvent(P.stream, h->fork, 0) != cudaSuccess) return TIKH_ECUDA;
    for (int w = 0; w < g->waves; ++w) {
      const int64_t off = (int64_t)w * g->W;
      const int nb = (int)std::min<int64_t>(g->W, (int64_t)g->items.size() - off);
      P.items = P.items_base + off;
      P.lam = P.lam_base + off;
      P.keep_status = w > 0;  // the status word collects every wave's failures
      int rc = enqueue_solve(P, 0, nb);
      if (rc) return rc;
      nl += P.launches;
    }
    if (cudaEventRecord(g->done, P.stream) != cudaSuccess || cudaStreamWaitEvent(h->stream, g->done, 0) != cudaSuccess)
      return TIKH_ECUDA;
  }
  h->launches = nl;
  return TIKH_OK;
}

void batch_drop_graph(tikh_batch_plan h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
}

// wave w of group g on the group's stream: its solve, or the replay of its captured graph
int wave_capture(BatchGroup* g, int w) {
  Plan& P = g->P;
  const int64_t off = (int64_t)w * g->W;
  const int nb = (int)std::min<int64_t>(g->W, (int64_t)g->items.size() - off);
  P.items = P.items_base + off;
  P.lam = P.lam_base + off;
  P.keep_status = w > 0;
  cudaGraph_t gr = nullptr;
  if (cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return TIKH_ECUDA;
  }
  int rc = enqueue_solve(P, 0, nb);
  cudaError_t ce = cudaStreamEndCapture(P.stream, &gr);
  cudaGraphExec_t ex = nullptr;
  if (!rc && ce == cudaSuccess && gr && cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) ex = nullptr;
  if (gr) cudaGraphDestroy(gr);
  cudaGetLastError();
  if (rc) return rc;
  if (!ex) return TIKH_ECUDA;
  g->graphs[(size_t)w] = ex;
  return TIKH_OK;
}

// With opts.graph every wave of every group is one captured graph (each about the size of one solve's
// schedule), replayed in order on the group's stream between the fork and join events; the first call
// captures them.  Without it (or while profiling) the waves are stream launches.
int batch_run(tikh_batch_plan h) {
  h->last.graph = 0;
  if (!h->opts.graph || h->prof) return batch_enqueue(h);
  int64_t nl = 0;
  for (BatchGroup* g : h->groups) {
    if ((int)g->graphs.size() != g->waves) {
      g->graphs.assign((size_t)g->waves, nullptr);
      for (int w = 0; w < g->waves; ++w) {
        int rc = wave_capture(g, w);
        if (rc) {  // capture not possible here: plain stream launches from now on
          drop_wave_graphs(g);
          for (BatchGroup* q : h->groups) drop_wave_graphs(q);
          h->opts.graph = 0;
          return batch_enqueue(h);
        }
      }
    }
  }
  if (cudaEventRecord(h->fork, h->stream) != cudaSuccess) return TIKH_ECUDA;
  for (BatchGroup* g : h->groups) {
    Plan& P = g->P;
    if (cudaStreamWaitEvent(P.stream, h->fork, 0) != cudaSuccess) return TIKH_ECUDA;
    for (int w = 0; w < g->waves; ++w) {
      if (cudaGraphLaunch(g->graphs[(size_t)w], P.stream) != cudaSuccess) return TIKH_ECUDA;
      nl += P.launches;
    }
    // the group's last-wave size for the status read
    P.nb = (int)std::min<int64_t>(g->W, (int64_t)g->items.size() - (int64_t)(g->waves - 1) * g->W);
    if (cudaEventRecord(g->done, P.stream) != cudaSuccess || cudaStreamWaitEvent(h->stream, g->done, 0) != cudaSuccess)
      return TIKH_ECUDA;
  }
  h->launches = nl;
  h->last.graph = 1;
  return TIKH_OK;
}

}  // namespace

extern "C" {

int tikh_plan_create(tikh_plan* out, int64_t m, int64_t n, int dtype, int prec, const tikh_opts* opts, void* stream) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (m < 1 || n < 1 || (dtype != TIKH_R64 && dtype != TIKH_C128) || !valid_prec(prec)) return TIKH_EINVAL;
  tikh_opts o{32, 0, 0, 1e-8, 4096, 0, 1, 0, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (!valid_opts(o)) return TIKH_EINVAL;
  const int64_t cm = std::max(m, n), cn = std::min(m, n);
  int64_t N, M;
  int p;
  if (!alg2(cm, cn, o, N, M, p)) return TIKH_EINVAL;
  tikh_plan h = new (std::nothrow) tikh_plan_s;
  if (!h) return TIKH_ENOMEM;
  int err = plan_setup(h->P, std::vector<Shape>(1, core_shape(m, n, N)), N, M, p, dtype, prec, o,
                       (cudaStream_t)stream, o.batch);
  if (err) {
    delete h;
    return err;
  }
  size_t es = dtype == TIKH_C128 ? 16 : 8;
  h->P.d_in = dalloc(h->P, es * (size_t)(2 * m + 2 * n) + 64, err);
  if (err) {
    free_plan(h->P);
    delete h;
    return err;
  }
  *out = h;
  return TIKH_OK;
}

int tikh_plan_create_gramian(tikh_plan* out, int64_t n, int64_t p, int dtype, int prec, const tikh_opts* opts,
                             void* stream) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (n < 1 || p < 1 || (dtype != TIKH_R64 && dtype != TIKH_C128) || !valid_prec(prec)) return TIKH_EINVAL;
  tikh_opts o{32, 0, 0, 1e-8, 4096, 0, 1, 0, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (!valid_opts(o)) return TIKH_EINVAL;
  // Sec. 3.4: the first block row has q = max(n, p) extension rows at k = 1, so N >= q + n - 1; L takes
  // T's place, with extension k = N - (p + n - 1)
  int64_t N, M;
  int pp;
  if (!alg2(std::max(n, p), n, o, N, M, pp)) return TIKH_EINVAL;
  Shape sh;
  sh.m = p;
  sh.n = n;
  sh.cm = p;
  sh.cn = n;
  sh.k = N - (p + n - 1);
  sh.dual = 0;
  tikh_plan h = new (std::nothrow) tikh_plan_s;
  if (!h) return TIKH_ENOMEM;
  h->P.gram = 1;
  int err = plan_setup(h->P, std::vector<Shape>(1, sh), N, M, pp, dtype, prec, o, (cudaStream_t)stream, o.batch);
  if (err) {
    delete h;
    return err;
  }
  *out = h;
  return TIKH_OK;
}

// the general problem (Sec. 3.2): (T^H T + L^H L) x = y with T m x n and L pl x n; three condition sets per
// node and a 7 x 7 basis; N >= max(m, pl) + n - 1 by Algorithm 2 with three sets; FP64 stages only
int tikh_plan_create_general(tikh_plan* out, int64_t m, int64_t n, int64_t pl, int dtype, const tikh_opts* opts,
                             void* stream) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (m < 1 || n < 1 || pl < 1 || (dtype != TIKH_R64 && dtype != TIKH_C128)) return TIKH_EINVAL;
  // defaults: leaves of 3 M <= 30 conditions; difficult-point threshold 1e-12 (deferring the conditions
  // whose best ratio lies in [1e-12, 1e-8) and processing them against B* costs accuracy here)
  tikh_opts o{30, 0, 0, 1e-12, 4096, 0, 1, 0, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  if (!valid_opts(o)) return TIKH_EINVAL;
  int64_t N, M;
  int pp;
  if (!alg2_sets(std::max(m, pl) + n - 1, 3, 42, o, N, M, pp)) return TIKH_EINVAL;
  Shape sh;
  sh.m = m;
  sh.n = n;
  sh.cm = m;
  sh.cn = n;
  sh.k = N - (m + n - 1);
  sh.pl = pl;
  sh.kl = N - (pl + n - 1);
  sh.dual = 0;
  tikh_plan h = new (std::nothrow) tikh_plan_s;
  if (!h) return TIKH_ENOMEM;
  h->P.general = 1;
  h->P.w = 7;
  h->P.ns = 3;
  int err = plan_setup(h->P, std::vector<Shape>(1, sh), N, M, pp, dtype, TIKH_PREC_FP64, o, (cudaStream_t)stream,
                       o.batch);
  if (err) {
    delete h;
    return err;
  }
  *out = h;
  return TIKH_OK;
}

static int general_run(tikh_plan h, int batch, const void* col, int64_t col_stride, const void* row,
                       int64_t row_stride, const void* lcol, int64_t lcol_stride, const void* lrow,
                       int64_t lrow_stride, const void* rhs, int64_t rhs_stride, void* x, int64_t x_stride,
                       int rhs_is_y) {
  if (!h || !h->P.general || !col || !row || !lcol || !lrow || !rhs || !x || batch < 1 || batch > h->P.batch_max)
    return TIKH_EINVAL;
  Plan& P = h->P;
  // an input stride is 0 (one array shared by the batch) or at least the array's length
  auto bad_stride = [](int64_t st, int64_t len) { return st < 0 || (st > 0 && st < len); };
  if (batch > 1 && (bad_stride(col_stride, P.m) || bad_stride(row_stride, P.n) || bad_stride(lcol_stride, P.pl) ||
                    bad_stride(lrow_stride, P.n) || bad_stride(rhs_stride, rhs_is_y ? P.n : P.m) || x_stride < P.n))
    return TIKH_EINVAL;
  const size_t es = P.dtype == TIKH_C128 ? 16 : 8;
  std::vector<ItemDev> items;
  items.reserve((size_t)batch);
  for (int i = 0; i < batch; ++i) {
    ItemDev it = make_item(P.shapes[0], (const char*)col + es * (size_t)(i * col_stride),
                           (const char*)row + es * (size_t)(i * row_stride),
                           (const char*)rhs + es * (size_t)(i * rhs_stride), (char*)x + es * (size_t)(i * x_stride));
    it.lcol = (const char*)lcol + es * (size_t)(i * lcol_stride);
    it.lrow = (const char*)lrow + es * (size_t)(i * lrow_stride);
    it.pl = P.shapes[0].pl;
    it.kl = P.shapes[0].kl;
    items.push_back(it);
  }
  const std::vector<double> zeros((size_t)batch, 0.0);  // the regularisation is in L
  return solve_with_retry(P, items, zeros.data(), rhs_is_y, nullptr, nullptr, 0);
}

int tikh_solve_general(tikh_plan h, const void* col, const void* row, const void* lcol, const void* lrow,
                       const void* b, void* x) {
  return general_run(h, 1, col, 0, row, 0, lcol, 0, lrow, 0, b, 0, x, 0, 0);
}

int tikh_solve_general_normal(tikh_plan h, const void* col, const void* row, const void* lcol, const void* lrow,
                              const void* y, void* x) {
  return general_run(h, 1, col, 0, row, 0, lcol, 0, lrow, 0, y, 0, x, 0, 1);
}

int tikh_solve_general_strided(tikh_plan h, int batch, const void* col, int64_t col_stride, const void* row,
                               int64_t row_stride, const void* lcol, int64_t lcol_stride, const void* lrow,
                               int64_t lrow_stride, const void* b, int64_t b_stride, void* x, int64_t x_stride) {
  return general_run(h, batch, col, col_stride, row, row_stride, lcol, lcol_stride, lrow, lrow_stride, b, b_stride, x,
                     x_stride, 0);
}

int tikh_solve_gramian(tikh_plan h, const void* g, const void* lcol, const void* lrow, const void* y, void* x) {
  if (!h || !g || !lcol || !lrow || !y || !x || !h->P.gram) return TIKH_EINVAL;
  std::vector<ItemDev> it = single(h->P, lcol, lrow, y, x);
  it[0].gram = g;
  const double zero = 0.0;  // the regularisation is in L
  return solve_with_retry(h->P, it, &zero, 1, nullptr, nullptr, 0);
}

int tikh_solve(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda) || h->P.gram || h->P.general) return TIKH_EINVAL;
  return solve_with_retry(h->P, single(h->P, col, row, b, x), &lambda, 0, nullptr, nullptr, 0);
}

int tikh_solve_async(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda) || h->P.gram || h->P.general) return TIKH_EINVAL;
  Plan& P = h->P;
  P.items = P.items_base;
  P.lam = P.lam_base;
  P.keep_status = false;
  std::vector<ItemDev> it = single(P, col, row, b, x);
  int rc = stage_items(P, it.data(), &lambda, 1, 0);
  return rc ? rc : enqueue_any(P, 0, 1);
}

int tikh_solve_normal(tikh_plan h, const void* col, const void* row, const void* y, double lambda, void* x) {
  if (!h || !col || !row || !y || !x || !valid_lambda(lambda) || h->P.gram || h->P.general || h->P.dual)
    return TIKH_EINVAL;
  return solve_with_retry(h->P, single(h->P, col, row, y, x), &lambda, 1, nullptr, nullptr, 0);
}

int tikh_solve_strided(tikh_plan h, int batch, const void* col, int64_t col_stride, const void* row,
                       int64_t row_stride, const void* b, int64_t b_stride, const double* lambdas, void* x,
                       int64_t x_stride) {
  if (!h || !col || !row || !b || !x || !lambdas || batch < 1 || batch > h->P.batch_max || h->P.gram || h->P.general)
    return TIKH_EINVAL;
  if (col_stride < 0 || row_stride < 0 || b_stride < 0 || (batch > 1 && x_stride < h->P.n)) return TIKH_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!valid_lambda(lambdas[i])) return TIKH_EINVAL;
  const size_t es = h->P.dtype == TIKH_C128 ? 16 : 8;
  std::vector<ItemDev> items;
  items.reserve((size_t)batch);
  for (int i = 0; i < batch; ++i)
    items.push_back(make_item(h->P.shapes[0], (const char*)col + es * (size_t)(i * col_stride),
                              (const char*)row + es * (size_t)(i * row_stride), (const char*)b + es * (size_t)(i * b_stride),
                              (char*)x + es * (size_t)(i * x_stride)));
  return solve_with_retry(h->P, items, lambdas, 0, nullptr, nullptr, 0);
}

// the adjoint of `batch` problems: g = A^{-1} dL/dx by the superfast solve (items carry col, row and dL/dx),
// then the gradient transforms; dL/dlambda of each problem to the host array dlam
static int grad_run(Plan& P, const std::vector<ItemDev>& items, const double* lams, const void* x, int64_t x_stride,
                    const void* b, int64_t b_stride, void* dcol, void* drow, void* db, int64_t out_col_stride,
                    int64_t out_row_stride, int64_t out_b_stride, double* dlam) {
  if (P.dual || P.gram || P.general) return TIKH_EINVAL;  // the adjoint is implemented for the l2 problem, m >= n
  const int nb = (int)items.size();
  int err = 0;
  if (!P.gbuf || !P.gdl) {  // adjoint workspace, allocated by the first gradient call (again after a failure)
    if (!P.gbuf) P.gbuf = (cd*)dalloc(P, sizeof(cd) * (size_t)(4 * P.N + 2 * P.cm) * (size_t)P.batch_max, err);
    if (!P.gdl) P.gdl = (double*)dalloc(P, sizeof(double) * (size_t)P.batch_max, err);
    if (err) return err;
  }
  P.items = P.items_base;
  P.lam = P.lam_base;
  P.keep_status = false;
  int r = stage_items(P, items.data(), lams, nb, 0);
  if (r) return r;
  int64_t nl = 0;
  if ((r = enqueue_prologue(P, 1, nb, nl)) < 0) return r;  // right-hand side y = dL/dx
  if ((r = enqueue_core_refined(P, nl)) < 0) return r;     // g = A^{-1} dL/dx
  if ((r = launch_grad(P, x, x_stride, b, b_stride, dcol, out_col_stride, drow, out_row_stride, db, out_b_stride, P.gdl,
                       P.gbuf)) < 0)
    return r;
  nl += r;
  P.launches = nl;
  if (cudaMemcpyAsync(dlam, P.gdl, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
    return TIKH_ECUDA;
  return sync_status(P);
}

int tikh_solve_grad(tikh_plan h, const void* col, const void* row, const void* b, double lambda, const void* x,
                    const void* dLdx, void* dLdcol, void* dLdrow, void* dLdb, double* dLdlambda) {
  if (!h || !col || !row || !b || !x || !dLdx || !dLdcol || !dLdrow || !dLdb || !dLdlambda || !valid_lambda(lambda))
    return TIKH_EINVAL;
  return grad_run(h->P, single(h->P, col, row, dLdx, nullptr), &lambda, x, 0, b, 0, dLdcol, dLdrow, dLdb, 0, 0, 0,
                  dLdlambda);
}

int tikh_solve_grad_strided(tikh_plan h, int batch, const void* col, int64_t col_stride, const void* row,
                            int64_t row_stride, const void* b, int64_t b_stride, const double* lambdas, const void* x,
                            int64_t x_stride, const void* dLdx, int64_t dLdx_stride, void* dLdcol, void* dLdrow,
                            void* dLdb, double* dLdlambda) {
  if (!h || !col || !row || !b || !x || !dLdx || !dLdcol || !dLdrow || !dLdb || !dLdlambda || !lambdas || batch < 1 ||
      batch > h->P.batch_max)
    return TIKH_EINVAL;
  Plan& P = h->P;
  if (col_stride < P.m || row_stride < P.n || b_stride < P.m || x_stride < P.n || dLdx_stride < P.n) return TIKH_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!valid_lambda(lambdas[i])) return TIKH_EINVAL;
  const size_t es = P.dtype == TIKH_C128 ? 16 : 8;
  std::vector<ItemDev> items;
  for (int i = 0; i < batch; ++i)
    items.push_back(make_item(P.shapes[0], (const char*)col + es * (size_t)(i * col_stride),
                              (const char*)row + es * (size_t)(i * row_stride),
                              (const char*)dLdx + es * (size_t)(i * dLdx_stride), nullptr));
  return grad_run(P, items, lambdas, x, x_stride, b, b_stride, dLdcol, dLdrow, dLdb, P.m, P.n, P.m, dLdlambda);
}

int tikh_solve_host(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda) || h->P.gram || h->P.general) return TIKH_EINVAL;
  Plan& P = h->P;
  size_t es = P.dtype == TIKH_C128 ? 16 : 8;
  char* base = (char*)P.d_in;
  char* dcol = base;
  char* drow = dcol + es * P.m;
  char* db = drow + es * P.n;
  char* dx = db + es * P.m;
  if (cudaMemcpyAsync(dcol, col, es * P.m, cudaMemcpyHostToDevice, P.stream) != cudaSuccess ||
      cudaMemcpyAsync(drow, row, es * P.n, cudaMemcpyHostToDevice, P.stream) != cudaSuccess ||
      cudaMemcpyAsync(db, b, es * P.m, cudaMemcpyHostToDevice, P.stream) != cudaSuccess)
    return TIKH_ECUDA;
  return solve_with_retry(P, single(P, dcol, drow, db, dx), &lambda, 0, x, dx, es * P.n);
}

int tikh_batch_plan_create(tikh_batch_plan* out, int nprob, const int64_t* m, const int64_t* n, int nlambda, int dtype,
                           int prec, const tikh_opts* opts, int64_t max_workspace_bytes, void* stream) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (nprob < 1 || nlambda < 1 || !m || !n || (int64_t)nprob * nlambda > (1LL << 30) ||
      (dtype != TIKH_R64 && dtype != TIKH_C128) || !valid_prec(prec) || max_workspace_bytes < 0)
    return TIKH_EINVAL;
  tikh_opts o{32, 0, 0, 1e-8, 4096, 0, 1, 0, 0, 0, 0, 0.0, 0, 0};
  if (opts) o = *opts;
  o.batch = 1;
  if (!valid_opts(o)) return TIKH_EINVAL;
  for (int i = 0; i < nprob; ++i)
    if (m[i] < 1 || n[i] < 1) return TIKH_EINVAL;
  tikh_batch_plan h = new (std::nothrow) tikh_batch_plan_s;
  if (!h) return TIKH_ENOMEM;
  h->nprob = nprob;
  h->nlambda = nlambda;
  h->dtype = dtype;
  h->opts = o;
  h->stream = (cudaStream_t)stream;
  h->m.assign(m, m + nprob);
  h->n.assign(n, n + nprob);
  h->group_of.assign((size_t)nprob, -1);
  // groups: problems whose core problems share (N, M, p) and the m < n form
  struct Key { int64_t N, M; int p, dual; };
  std::vector<Key> keys;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < nprob; ++i) {
    const int64_t cm = std::max(m[i], n[i]), cn = std::min(m[i], n[i]);
    int64_t N, M;
    int p;
    if (!alg2(cm, cn, o, N, M, p)) { batch_free(h); return TIKH_EINVAL; }
    const int dual = m[i] < n[i] ? 1 : 0;
    size_t g = 0;
    while (g < keys.size() && !(keys[g].N == N && keys[g].M == M && keys[g].p == p && keys[g].dual == dual)) ++g;
    if (g == keys.size()) { keys.push_back(Key{N, M, p, dual}); members.emplace_back(); }
    members[g].push_back(i);
    h->group_of[(size_t)i] = (int)g;
  }
  // per-item workspace of each group, from a one-item plan of its shapes; then the wave size W of every
  // group scaled so that the groups together fit the workspace budget
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); batch_free(h); return TIKH_ECUDA; }
  const double budget = max_workspace_bytes > 0 ? (double)max_workspace_bytes : 0.6 * (double)free_b;
  std::vector<double> per_item(keys.size());
  std::vector<std::vector<Shape>> gshapes(keys.size());
  double need = 0.0;
  for (size_t g = 0; g < keys.size(); ++g) {
    for (int i : members[g]) {
      Shape sh = core_shape(m[i], n[i], keys[g].N);
      bool seen = false;
      for (const Shape& q : gshapes[g]) seen = seen || (q.m == sh.m && q.n == sh.n);
      if (!seen) gshapes[g].push_back(sh);
    }
    Plan probe;
    tikh_opts o1 = o;
    o1.batch = 1;
    int err = plan_setup(probe, gshapes[g], keys[g].N, keys[g].M, keys[g].p, dtype, prec, o1, h->stream, 1);
    if (err) { batch_free(h); return err; }
    per_item[g] = (double)probe.bytes;
    free_plan(probe);
    need += per_item[g] * (double)members[g].size() * nlambda;
  }
  const double scale = need > budget ? budget / need : 1.0;
  int err = 0;
  if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) err = TIKH_ECUDA;
  for (size_t g = 0; g < keys.size() && !err; ++g) {
    BatchGroup* G = new (std::nothrow) BatchGroup;
    if (!G) { err = TIKH_ENOMEM; break; }
    h->groups.push_back(G);
    for (int i : members[g])
      for (int l = 0; l < nlambda; ++l) G->items.push_back((int64_t)i * nlambda + l);
    const int64_t cnt = (int64_t)G->items.size();
    G->W = (int)std::max<int64_t>(1, std::min<int64_t>({cnt, (int64_t)(cnt * scale), 65535}));
    G->waves = (int)((cnt + G->W - 1) / G->W);
    cudaStream_t gs = nullptr;
    if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming) != cudaSuccess) {
      err = TIKH_ECUDA;
      if (gs) cudaStreamDestroy(gs);
      break;
    }
    G->P.stream = gs;
    tikh_opts og = o;
    og.batch = G->W;
    // the direct/FFT thresholds follow the group's item count, not its wave size, so an item's arithmetic
    // does not depend on the workspace budget
    int auto_prod, auto_eval;
    auto_thresholds(cnt, prec, auto_prod, auto_eval);
    if (og.prod_direct_max == 0) og.prod_direct_max = auto_prod;
    if (og.eval_direct_max == 0) og.eval_direct_max = auto_eval;
    err = plan_setup(G->P, gshapes[g], keys[g].N, keys[g].M, keys[g].p, dtype, prec, og, gs, cnt);
    if (err) G->P.stream = gs;  // destroyed by batch_free
  }
  if (err) {
    cudaGetLastError();
    batch_free(h);
    return err;
  }
  h->last.ngroups = (int)h->groups.size();
  for (BatchGroup* G : h->groups) {
    h->last.max_waves = std::max(h->last.max_waves, G->waves);
    h->last.workspace_bytes += G->P.bytes;
  }
  h->last.items = (int64_t)nprob * nlambda;
  h->last.rel_residual = -1.0;
  *out = h;
  return TIKH_OK;
}

int tikh_solve_batched(tikh_batch_plan h, int nprob, const int64_t* m, const int64_t* n, const void* const* col,
                       const void* const* row, const void* const* b, int nlambda, const double* lambdas,
                       void* const* x) {
  if (!h || !m || !n || !col || !row || !b || !lambdas || !x || nprob != h->nprob || nlambda != h->nlambda)
    return TIKH_EINVAL;
  for (int i = 0; i < nprob; ++i)
    if (m[i] != h->m[(size_t)i] || n[i] != h->n[(size_t)i] || !col[i] || !row[i] || !b[i]) return TIKH_EINVAL;
  for (int l = 0; l < nlambda; ++l)
    if (!valid_lambda(lambdas[l])) return TIKH_EINVAL;
  for (int64_t q = 0; q < (int64_t)nprob * nlambda; ++q)
    if (!x[q]) return TIKH_EINVAL;
  for (int attempt = 0;; ++attempt) {
    // item tables of every wave of every group (outside the graph), then the forked solve
    for (BatchGroup* G : h->groups) {
      std::vector<ItemDev> items;
      std::vector<double> lams;
      items.reserve(G->items.size());
      lams.reserve(G->items.size());
      for (int64_t id : G->items) {
        const int i = (int)(id / nlambda), l = (int)(id % nlambda);
        const Shape sh = core_shape(m[i], n[i], G->P.N);
        items.push_back(make_item(sh, col[i], row[i], b[i], x[id]));
        lams.push_back(lambdas[l]);
      }
      // the group's tables are written on the plan's stream, ahead of the fork that starts the group
      Plan& P = G->P;
      if (cudaMemcpyAsync(P.items_base, items.data(), sizeof(ItemDev) * items.size(), cudaMemcpyHostToDevice,
                          h->stream) != cudaSuccess ||
          cudaMemcpyAsync(P.lam_base, lams.data(), sizeof(double) * lams.size(), cudaMemcpyHostToDevice, h->stream) !=
              cudaSuccess)
        return TIKH_ECUDA;
    }
    int rc = batch_run(h);
    if (rc) return rc;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) { cudaGetLastError(); return TIKH_ECUDA; }
    int worst = TIKH_OK;
    bool degree = false;
    h->last.rel_residual = -1.0;
    h->last.n_difficult = 0;
    h->last.last_correction = -1.0;
    for (int k = 0; k < 4; ++k) h->last.model_flops[k] = h->last.model_flops_fp32[k] = 0.0;
    for (BatchGroup* G : h->groups) {
      if (h->prof) {  // the profiled group's events were recorded on the plan's stream
        cudaStream_t own = G->P.stream;
        G->P.stream = h->stream;
        int c = sync_status(G->P);
        G->P.stream = own;
        if (c == TIKH_EDEGREE) degree = true;
        else if (c && !worst) worst = c;
      } else {
        int c = sync_status(G->P);
        if (c == TIKH_EDEGREE) degree = true;
        else if (c && !worst) worst = c;
      }
      const tikh_stats& gl = G->P.last;
      h->last.rel_residual = std::max(h->last.rel_residual, gl.rel_residual);
      h->last.last_correction = std::max(h->last.last_correction, gl.last_correction);
      h->last.n_difficult += gl.n_difficult;
      const double cnt = (double)G->items.size();
      for (int k = 0; k < 4; ++k) {
        h->last.model_flops[k] += gl.model_flops[k] * cnt;
        h->last.model_flops_fp32[k] += gl.model_flops_fp32[k] * cnt;
      }
    }
    if (h->prof) {
      for (int k = 0; k < 4; ++k) {
        h->last.prof_kind_ms[k] = 0.0;
        h->last.prof_kind_count[k] = 0;
        for (BatchGroup* G : h->groups) {
          h->last.prof_kind_ms[k] += G->P.last.prof_kind_ms[k];
          h->last.prof_kind_count[k] += G->P.last.prof_kind_count[k];
        }
      }
    }
    h->last.kernel_launches = h->launches;
    if (worst) return worst;
    if (!degree) return TIKH_OK;
    if (attempt >= 3) return TIKH_EDEGREE;
    // a basis outgrew its planned transform: more degree slack for every group, re-plan, re-run
    batch_drop_graph(h);
    for (BatchGroup* G : h->groups) {
      drop_wave_graphs(G);
      G->P.slack_mult *= 16;
      drop_graph(G->P);
      if ((rc = make_schedule(G->P))) return rc;
    }
    h->last.retries = attempt + 1;
  }
}

int tikh_batch_set_profiling(tikh_batch_plan h, int flags) {
  if (!h || flags < 0 || flags > 3) return TIKH_EINVAL;
  h->prof = flags;
  for (BatchGroup* G : h->groups)
    set_profiling(G->P, flags);
  for (int k = 0; k < 4; ++k) {
    h->last.prof_kind_ms[k] = 0.0;
    h->last.prof_kind_count[k] = 0;
  }
  return TIKH_OK;
}

int tikh_batch_get_stats(tikh_batch_plan h, tikh_batch_stats* out) {
  if (!h || !out) return TIKH_EINVAL;
  *out = h->last;
  out->workspace_bytes = 0;
  for (BatchGroup* G : h->groups) out->workspace_bytes += G->P.bytes;
  return TIKH_OK;
}

void tikh_batch_plan_destroy(tikh_batch_plan h) {
  if (h) batch_free(h);
}

int tikh_sync(tikh_plan h) {
  if (!h) return TIKH_EINVAL;
  return sync_status(h->P);
}

int tikh_get_difficult(tikh_plan h, int64_t* ids, int64_t cap, int64_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !ids)) return TIKH_EINVAL;
  Plan& P = h->P;
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) { cudaGetLastError(); return TIKH_ECUDA; }
  int nd = 0;
  if (cudaMemcpy(&nd, P.ndiff, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TIKH_ECUDA;
  *count = nd;
  const int64_t stored = std::min<int64_t>(std::min<int64_t>(nd, P.opts.max_difficult), cap);
  if (stored > 0 && cudaMemcpy(ids, P.diff, sizeof(int64_t) * (size_t)stored, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TIKH_ECUDA;
  return TIKH_OK;
}

int tikh_get_stats(tikh_plan h, tikh_stats* out) {
  if (!h || !out) return TIKH_EINVAL;
  *out = h->P.last;
  out->workspace_bytes = h->P.bytes;
  return TIKH_OK;
}

int tikh_set_profiling(tikh_plan h, int flags) {
  if (!h || flags < 0 || flags > 3) return TIKH_EINVAL;
  set_profiling(h->P, flags);
  return TIKH_OK;
}

void tikh_plan_destroy(tikh_plan h) {
  if (!h) return;
  free_plan(h->P);
  delete h;
}

// ---- one solver for many right-hand sides (csrc/inverse.cu) ----

struct tikh_inverse_s {
  Plan* P = nullptr;  // the plan it was built with (not owned): FFT tables, stream
  InvWork w;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t launches = 0;  // kernels of the last create or apply
};

static void inverse_free(tikh_inverse v) {
  for (void* p : v->allocs) cudaFree(p);
  delete v;
}

int tikh_inverse_create(tikh_inverse* out, tikh_plan h, const void* col, const void* row, double lambda,
                        int max_rhs) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (!h || !col || !row || !valid_lambda(lambda) || max_rhs < 1 || max_rhs > 4096) return TIKH_EINVAL;
  Plan& P = h->P;
  if (P.gram || P.general || P.dual || P.shapes.size() != 1) return TIKH_EINVAL;
  // the batched four-step passes index batch x L2 transforms with int
  const FftPlan& F0 = P.ffts[P.fft_of_len.at(P.N)];
  if (F0.four && (int64_t)std::max(4 * max_rhs, 8) * std::max(F0.L1, F0.L2) >= (int64_t)1 << 30) return TIKH_EINVAL;
  tikh_inverse v = new (std::nothrow) tikh_inverse_s;
  if (!v) return TIKH_ENOMEM;
  v->P = &P;
  InvWork& w = v->w;
  w.m = P.m;
  w.n = P.n;
  w.N = P.N;
  w.dtype = P.dtype;
  w.lam = lambda;
  w.R = max_rhs;
  int err = 0;
  auto al = [&](size_t bytes) -> void* {
    if (err) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      err = TIKH_ENOMEM;
      return nullptr;
    }
    v->allocs.push_back(p);
    v->bytes += (int64_t)bytes;
    return p;
  };
  const size_t N = (size_t)P.N, n = (size_t)P.n, m = (size_t)P.m, R = (size_t)max_rhs, c = sizeof(cd);
  const size_t es = P.dtype == TIKH_C128 ? 16 : 8;
  w.spec = (cd*)al(c * 9 * N);
  w.gen = (cd*)al(c * 8 * n);
  w.Ae = (cd*)al(c * 2 * n);
  w.rhs8 = al(es * 8 * n);
  w.sol8 = al(es * 8 * n);
  w.Y = (cd*)al(c * std::max<size_t>(R, 2) * N);
  w.C = (cd*)al(c * 4 * R * N);
  w.G = (cd*)al(c * 4 * R * N);
  w.tmp = (cd*)al(c * std::max<size_t>(4 * R, 8) * N);
  w.y = (cd*)al(c * R * n);
  w.x = (cd*)al(c * R * n);
  w.r = (cd*)al(c * R * n);
  w.u = (cd*)al(c * R * m);
  if (err) {
    inverse_free(v);
    return err;
  }
  int rc = launch_inv_prepare(F0, w, col, row, P.stream);
  if (rc < 0) {
    inverse_free(v);
    return rc;
  }
  int64_t nl = rc;
  // the eight solves X v_i (normal form), as batches of the plan's size
  for (int i0 = 0; i0 < 8; i0 += P.batch_max) {
    const int cnt = std::min(8 - i0, P.batch_max);
    std::vector<ItemDev> items;
    for (int i = i0; i < i0 + cnt; ++i)
      items.push_back(make_item(P.shapes[0], col, row, (const char*)w.rhs8 + es * n * (size_t)i,
                                (char*)w.sol8 + es * n * (size_t)i));
    const std::vector<double> lams((size_t)cnt, lambda);
    if ((rc = solve_with_retry(P, items, lams.data(), 1, nullptr, nullptr, 0))) {
      inverse_free(v);
      return rc;
    }
    nl += P.last.kernel_launches;
  }
  // a re-plan inside the solves may have grown P.ffts: look the length-N transform up again
  if ((rc = launch_inv_terms(P.ffts[P.fft_of_len.at(P.N)], w, P.stream)) < 0) {
    inverse_free(v);
    return rc;
  }
  v->launches = nl + rc;
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) {
    cudaGetLastError();
    inverse_free(v);
    return TIKH_ECUDA;
  }
  *out = v;
  return TIKH_OK;
}

int tikh_inverse_apply(tikh_inverse v, int nrhs, const void* b, int64_t b_stride, void* x, int64_t x_stride,
                       int normal, int refine_steps) {
  if (!v || !b || !x || nrhs < 1 || refine_steps < 0 || refine_steps > 16 || (normal != 0 && normal != 1))
    return TIKH_EINVAL;
  InvWork& w = v->w;
  if (nrhs > 1 && (b_stride < (normal ? w.n : w.m) || x_stride < w.n)) return TIKH_EINVAL;
  Plan& P = *v->P;
  const FftPlan& F = P.ffts[P.fft_of_len.at(w.N)];
  const size_t es = w.dtype == TIKH_C128 ? 16 : 8;
  int64_t nl = 0;
  for (int c0 = 0; c0 < nrhs; c0 += w.R) {
    const int nb = std::min(w.R, nrhs - c0);
    const int rc = launch_inv_apply(F, w, nb, (const char*)b + es * (size_t)c0 * (size_t)b_stride, b_stride, normal,
                                    refine_steps, (char*)x + es * (size_t)c0 * (size_t)x_stride, x_stride, P.stream);
    if (rc < 0) return rc;
    nl += rc;
  }
  v->launches = nl;
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) {
    cudaGetLastError();
    return TIKH_ECUDA;
  }
  return TIKH_OK;
}

int tikh_inverse_generators(tikh_inverse v, void* out) {
  if (!v || !out) return TIKH_EINVAL;
  if (cudaMemcpyAsync(out, v->w.gen, sizeof(cd) * 8 * (size_t)v->w.n, cudaMemcpyDeviceToDevice, v->P->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(v->P->stream) != cudaSuccess) {
    cudaGetLastError();
    return TIKH_ECUDA;
  }
  return TIKH_OK;
}

int tikh_inverse_info(tikh_inverse v, int64_t* kernel_launches, int64_t* workspace_bytes) {
  if (!v || !kernel_launches || !workspace_bytes) return TIKH_EINVAL;
  *kernel_launches = v->launches;
  *workspace_bytes = v->bytes;
  return TIKH_OK;
}

void tikh_inverse_destroy(tikh_inverse v) {
  if (v) inverse_free(v);
}

const char* tikh_strerror(int s) {
  switch (s) {
    case TIKH_OK: return "ok";
    case TIKH_EINVAL: return "invalid argument";
    case TIKH_ENOMEM: return "out of device memory";
    case TIKH_ECUDA: return "CUDA runtime error";
    case TIKH_ENUMERIC: return "numerical failure (degree pattern or non-finite value)";
    case TIKH_EDIFFICULT: return "too many difficult points";
    case TIKH_ENOTCONVERGED: return "refinement did not converge";
    case TIKH_ETIMEOUT: return "device wait timed out";
    case TIKH_EDEGREE: return "basis degree exceeded the planned transform length";
    default: return "unknown status";
  }
}

}  // extern "C"
