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

int fft_index(Plan& P, int64_t L, int& err) {
  auto it = P.fft_of_len.find(L);
  if (it != P.fft_of_len.end()) return it->second;
  FftPlan f;
  f.L = L;
  if (L <= FFT_TILE_MAX) {
    if (!fft_factor((int)L, f.d1)) { err = TIKH_EINVAL; return -1; }
    f.d1.tw = twiddle(P, L, err);
  } else {
    int64_t L1, L2;
    if (!fft_split(L, L1, L2)) { err = TIKH_EINVAL; return -1; }
    f.four = true;
    f.L1 = L1;
    f.L2 = L2;
    fft_factor((int)L1, f.d1);
    fft_factor((int)L2, f.d2);
    f.d1.tw = twiddle(P, L1, err);
    f.d2.tw = twiddle(P, L2, err);
    f.twL = twiddle(P, L, err);
  }
  if (err) return -1;
  P.ffts.push_back(f);
  P.fft_of_len[L] = (int)P.ffts.size() - 1;
  return (int)P.ffts.size() - 1;
}

// same bound as the device: tau-degree bound for pivoted columns, accumulation bound otherwise
int entry_bound_host(const int* din, const int* dout, int i, int j) {
  int amax = 0;
  bool have = false;
  for (int c = 0; c < 5; ++c)
    if (dout[c] > din[c]) { amax = have ? std::max(amax, dout[c]) : dout[c]; have = true; }
  if (dout[j] > din[j]) return dout[j] - din[i];
  int acc = have ? amax - din[i] : -1;
  if (i == j && acc < 0) acc = 0;
  return std::min(acc, dout[j] - din[i]);
}

void waterfill(int* d, int64_t C) {
  for (int64_t c = 0; c < C; ++c) {
    int j = 0;
    for (int i = 1; i < 5; ++i)
      if (d[i] < d[j]) j = i;
    d[j] += 1;
  }
}

void build_steps(Plan& P, int depth, int64_t a, int64_t s, int64_t L, int side, int* sd, uint64_t& pending,
                 int64_t slack, int& err) {
  if (err) return;
  if (depth == P.p) {
    Step st{STEP_LEAF, depth, side, a, s, L, -1, 0, pending};
    pending = 0;
    waterfill(sd, 4 * L);
    P.sched.push_back(st);
    return;
  }
  int din[5];
  memcpy(din, sd, sizeof(din));
  pending |= (1ULL << depth);
  build_steps(P, depth + 1, a, 2 * s, L / 2, 0, sd, pending, slack, err);
  Step ev{STEP_EVAL, depth, side, a, s, L, fft_index(P, L / 2, err), 0, 0};
  P.sched.push_back(ev);
  P.Lrmax = std::max(P.Lrmax, L / 2);
  build_steps(P, depth + 1, a + s, 2 * s, L / 2, 1, sd, pending, slack, err);
  int D = -1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) D = std::max(D, entry_bound_host(din, sd, i, j));
  // the product of the bases of 4L conditions has degree <= 4L whatever the tau-degree bound and the
  // slack say, and each child's stored entries are at most 2L + 1 long (they are trimmed to the same
  // kind of bound), which the transform must hold
  int64_t Pn = smooth_at_least(std::max<int64_t>(2 * L + 1, std::min<int64_t>((int64_t)D + 1 + slack, 4 * L + 1)));
  Step pr{STEP_PROD, depth, side, a, s, L, fft_index(P, Pn, err), Pn, 0};
  P.sched.push_back(pr);
  P.Pmax = std::max(P.Pmax, Pn);
}

// (re)build the schedule, the product scratch and the basis buffers for the current slack
int make_schedule(Plan& P) {
  int err = 0;
  const size_t nb = (size_t)P.batch_max;
  P.sched.clear();
  int sd[5] = {-(int)(P.cn - 1), -(int)(P.cm - 1), -(int)(P.cm + P.k - 2), -(int)(P.cn + P.k - 2), 0};
  uint64_t pending = 0;
  int64_t oldP = P.Pmax;
  int64_t slack = (int64_t)P.slack_mult * (P.k + 2 * P.M + 4);
  build_steps(P, 0, 0, 2, P.N / 2, 0, sd, pending, slack, err);
  if (err) return err;
  if (P.Pmax > oldP || !P.FA) {
    size_t n25 = 25 * (size_t)std::max<int64_t>(P.Pmax, 1) * nb;
    P.FA = (cd*)dalloc(P, sizeof(cd) * n25, err);
    P.FB = (cd*)dalloc(P, sizeof(cd) * n25, err);
    P.FC = (cd*)dalloc(P, sizeof(cd) * n25, err);
    P.ptmp = (cd*)dalloc(P, sizeof(cd) * 2 * n25, err);
  }
  // basis capacity per depth: a product's entries are at most P long (P exceeds every entry degree
  // bound of the node, which can exceed the node's condition count by the spread of delta_in);
  // leaves hold at most K + 1 coefficients; the root also absorbs the difficult points
  int64_t need[MAX_DEPTH] = {0};
  need[P.p] = 2 * P.M + 1;
  for (const Step& st : P.sched)
    if (st.kind == STEP_PROD) need[st.depth] = std::max(need[st.depth], st.P);
  need[0] += std::min(P.opts.max_difficult, 4096) + 2;
  for (int d = 0; d <= P.p && !err; ++d)
    for (int side = 0; side < (d == 0 ? 1 : 2); ++side) {
      BasisBuf& B = P.buf[d][side];
      if (B.cap >= need[d]) continue;
      B.cap = need[d];
      B.c = (cd*)dalloc(P, sizeof(cd) * 25 * (size_t)B.cap * nb, err);
      if (!B.len) B.len = (int*)dalloc(P, sizeof(int) * 32 * nb, err);
      if (!B.colmax) B.colmax = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * 8 * nb, err);
      if (d == 0) {
        P.dscr_stride = 5 * B.cap + P.opts.max_difficult;
        P.dscr = (cd*)dalloc(P, sizeof(cd) * (size_t)P.dscr_stride * nb, err);
      }
    }
  return err;
}

// the root cause first: a wait that gave up or a non-finite input invalidates everything after it; a
// full deferred list cannot be fixed by re-planning; a degree overflow (retried with more slack) can
// itself cause the final degree pattern or extraction to fail
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

int enqueue_prologue(Plan& P, const UserArrays& u, int rhs_is_y, const double* lams, int nb, int64_t& nl) {
  int r;
  if (nb < 1 || nb > P.batch_max) return TIKH_EINVAL;
  P.nb = nb;
  if (lams &&
      cudaMemcpyAsync(P.lam, lams, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, P.stream) != cudaSuccess)
    return TIKH_ECUDA;
  if (cudaMemsetAsync(P.status, 0, sizeof(int), P.stream) != cudaSuccess) return TIKH_ECUDA;
  ProfScope ps(P, 3);
  if ((r = launch_spectrum(P, u, rhs_is_y)) < 0) return r;
  nl += r;
  // for m < n the core problem (T T^H + lam I) v = b takes b itself as its right-hand side
  if ((r = launch_rhs(P, u, P.dual ? 1 : rhs_is_y)) < 0) return r;
  nl += r;
  return TIKH_OK;
}

int enqueue_solve(Plan& P, const UserArrays& u, int rhs_is_y, const double* lams, int nb) {
  int64_t nl = 0;
  int r;
  if ((r = enqueue_prologue(P, u, rhs_is_y, lams, nb, nl)) < 0) return r;
  if ((r = enqueue_core_refined(P, nl)) < 0) return r;
  {
    ProfScope ps(P, 3);
    if ((r = launch_output(P, P.xcore, u)) < 0) return r;
  }
  nl += r;
  P.launches = nl;
  return TIKH_OK;
}

bool same_args(const UserArrays& a, const UserArrays& b) {
  return a.col == b.col && a.row == b.row && a.rhs == b.rhs && a.x == b.x && a.col_stride == b.col_stride &&
         a.row_stride == b.row_stride && a.rhs_stride == b.rhs_stride && a.x_stride == b.x_stride;
}

void drop_graph(Plan& P) {
  if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
  P.graph_exec = nullptr;
  P.graph_nb = 0;
}

// the solve as a CUDA graph: lambda is uploaded outside the graph; the rest (status reset, transform,
// every node of the recursion, refinement, output) is captured once per argument set and replayed
int enqueue_solve_graph(Plan& P, const UserArrays& u, int rhs_is_y, const double* lams, int nb) {
  if (nb < 1 || nb > P.batch_max) return TIKH_EINVAL;
  if (cudaMemcpyAsync(P.lam, lams, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, P.stream) != cudaSuccess)
    return TIKH_ECUDA;
  if (!P.graph_exec || P.graph_nb != nb || P.graph_rhs_is_y != rhs_is_y || !same_args(P.graph_key, u)) {
    drop_graph(P);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();  // e.g. the legacy default stream, which cannot be captured
      P.opts.graph = 0;
      return enqueue_solve(P, u, rhs_is_y, nullptr, nb);
    }
    int rc = enqueue_solve(P, u, rhs_is_y, nullptr, nb);
    cudaError_t ce = cudaStreamEndCapture(P.stream, &g);
    if (rc || ce != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      P.opts.graph = 0;  // capture not possible here: plain stream launches from now on
      return rc ? rc : enqueue_solve(P, u, rhs_is_y, nullptr, nb);
    }
    ce = cudaGraphInstantiate(&P.graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      P.graph_exec = nullptr;
      P.opts.graph = 0;
      return enqueue_solve(P, u, rhs_is_y, nullptr, nb);
    }
    P.graph_key = u;
    P.graph_nb = nb;
    P.graph_rhs_is_y = rhs_is_y;
  }
  P.nb = nb;
  return cudaGraphLaunch(P.graph_exec, P.stream) == cudaSuccess ? TIKH_OK : TIKH_ECUDA;
}

int enqueue_any(Plan& P, const UserArrays& u, int rhs_is_y, const double* lams, int nb) {
  P.last.graph = 0;
  if (P.opts.graph && !P.prof_leaf) {
    int rc = enqueue_solve_graph(P, u, rhs_is_y, lams, nb);
    P.last.graph = P.graph_exec && P.opts.graph ? 1 : 0;
    return rc;
  }
  return enqueue_solve(P, u, rhs_is_y, lams, nb);
}

int sync_status(Plan& P) {
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) { cudaGetLastError(); return TIKH_ECUDA; }
  int st = 0;
  if (cudaMemcpy(&st, P.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TIKH_ECUDA;
  std::vector<int> nd(4 * (size_t)P.nb), dl(8 * (size_t)P.nb);
  cudaMemcpy(nd.data(), P.ndiff, sizeof(int) * nd.size(), cudaMemcpyDeviceToHost);
  cudaMemcpy(dl.data(), P.delta, sizeof(int) * dl.size(), cudaMemcpyDeviceToHost);
  int64_t total = 0;
  for (int b = 0; b < P.nb; ++b) total += nd[4 * b];
  P.last.n_difficult = total;
  memcpy(P.last.delta, dl.data(), sizeof(int) * 5);
  P.last.jstar = -1;
  for (int j = 0; j < 5; ++j)
    if (dl[j] == 0) P.last.jstar = j;
  P.last.kernel_launches = P.launches;
  P.last.refine_steps = P.opts.refine_steps;
  P.last.batch = P.nb;
  P.last.rel_residual = -1.0;
  if (P.opts.refine_steps > 0) {  // largest relative residual of the batch
    std::vector<double> nr(4 * (size_t)P.nb);
    cudaMemcpy(nr.data(), P.norms, sizeof(double) * nr.size(), cudaMemcpyDeviceToHost);
    double worst = 0.0;
    for (int b = 0; b < P.nb; ++b) {
      double v = nr[4 * b + 1] > 0.0 ? sqrt(nr[4 * b] / nr[4 * b + 1]) : sqrt(nr[4 * b]);
      worst = std::max(worst, v);
    }
    P.last.rel_residual = worst;
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
  return status_to_code(st);
}

int solve_with_retry(Plan& P, const UserArrays& u, int rhs_is_y, const double* lams, int nb, void* x_host,
                     size_t xbytes) {
  P.last.retries = 0;
  for (int attempt = 0;; ++attempt) {
    int rc = enqueue_any(P, u, rhs_is_y, lams, nb);
    if (rc) return rc;
    if (x_host && cudaMemcpyAsync(x_host, u.x, xbytes, cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
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

UserArrays single(const Plan& P, const void* col, const void* row, const void* rhs, void* x) {
  UserArrays u;
  u.col = col;
  u.row = row;
  u.rhs = rhs;
  u.x = x;
  return u;
}

}  // namespace

extern "C" {

int tikh_plan_create(tikh_plan* out, int64_t m, int64_t n, int dtype, int prec, const tikh_opts* opts, void* stream) {
  if (!out) return TIKH_EINVAL;
  *out = nullptr;
  if (m < 1 || n < 1 || (dtype != TIKH_R64 && dtype != TIKH_C128) || prec != TIKH_PREC_FP64) return TIKH_EINVAL;
  tikh_opts o{32, 0, 0, 1e-8, 4096, 0, 1, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (o.n_lim < 4 || o.n_lim > 64 || o.m_min < 0 || o.m_min > 32 || (o.fill != 0 && o.fill != 1) ||
      !(o.eps_diff >= 0.0) || o.max_difficult < 1 || o.max_difficult > (1 << 20) || o.refine_steps < 0 ||
      o.refine_steps > 8 || o.batch < 1 || o.batch > 65535 || (o.graph != 0 && o.graph != 1) ||
      o.prod_direct_max < 0 || o.prod_direct_max > 4096 || o.eval_direct_max < 0 || o.eval_direct_max > 4096 ||
      o.wait_polls < 0 || o.wait_polls > (1 << 30))
    return TIKH_EINVAL;
  tikh_plan h = new (std::nothrow) tikh_plan_s;
  if (!h) return TIKH_ENOMEM;
  Plan& P = h->P;
  P.m = m;
  P.n = n;
  P.dtype = dtype;
  P.opts = o;
  P.batch_max = o.batch;
  // direct vs FFT forms of steps 2 and 4: a single problem is latency-bound at small nodes (direct forms
  // spread over more SMs with short chains); a batch is FP64-throughput-bound, where the O(P^2) direct
  // product loses to the O(P log P) FFT product at much smaller P (measured on GB300)
  P.prod_direct_max = o.prod_direct_max > 0 ? o.prod_direct_max : (o.batch == 1 ? 360 : BATCH_PROD_DIRECT_MAX);
  P.eval_direct_max = o.eval_direct_max > 0 ? o.eval_direct_max : (o.batch == 1 ? 80 : BATCH_EVAL_DIRECT_MAX);
  P.wait_polls = o.wait_polls > 0 ? o.wait_polls : (1 << 24);
  P.stream = (cudaStream_t)stream;
  P.dual = m < n ? 1 : 0;
  P.cm = P.dual ? n : m;
  P.cn = P.dual ? m : n;
  // Algorithm 2 (reading: two condition sets, paired interleaving; M even, 7-smooth)
  int64_t Nt = P.cm + P.cn - 1, Mv = Nt;
  int pv = 0;
  while (2 * Mv > o.n_lim) { ++pv; Mv = (Mv + 1) / 2; }
  if (Mv % 2) ++Mv;
  if (Mv < o.m_min) Mv = o.m_min + (o.m_min % 2);
  while (!is_7smooth(Mv)) Mv += 2;
  P.M = Mv;
  P.p = pv;
  P.N = Mv << pv;
  P.k = P.N - Nt;
  if (pv >= MAX_DEPTH - 1 || 4 * (Mv / 2) > 64 || P.N > (int64_t)1 << 31) { delete h; return TIKH_EINVAL; }

  int err = 0;
  const size_t N = (size_t)P.N, nb = (size_t)P.batch_max;
  if (fft_index(P, P.N, err) < 0 && !err) err = TIKH_EINVAL;
  P.wN = P.twiddle_of_len[P.N];
  P.specT = (cd*)dalloc(P, sizeof(cd) * N * nb, err);
  P.work = (cd*)dalloc(P, sizeof(cd) * N * nb, err);
  P.work2 = (cd*)dalloc(P, sizeof(cd) * N * nb, err);
  P.ftmpN = (cd*)dalloc(P, sizeof(cd) * N * nb, err);
  P.R = (cd*)dalloc(P, sizeof(cd) * 10 * N * nb, err);
  P.Phi = (cd*)dalloc(P, sizeof(cd) * 10 * N * nb, err);
  P.delta = (int*)dalloc(P, sizeof(int) * 8 * nb, err);
  P.dstack = (int*)dalloc(P, sizeof(int) * 5 * MAX_DEPTH * nb, err);
  P.status = (int*)dalloc(P, sizeof(int) * 4, err);
  P.ndiff = (int*)dalloc(P, sizeof(int) * 4 * nb, err);
  P.bad = (int*)dalloc(P, sizeof(int) * nb, err);
  P.diff = (int64_t*)dalloc(P, sizeof(int64_t) * (size_t)o.max_difficult * nb, err);
  P.diffr = (cd*)dalloc(P, sizeof(cd) * 5 * (size_t)o.max_difficult * nb, err);
  P.dvals = (cd*)dalloc(P, sizeof(cd) * 25 * (size_t)o.max_difficult * nb, err);
  P.peak = (unsigned long long*)dalloc(P, sizeof(unsigned long long) * nb, err);
  P.lam = (double*)dalloc(P, sizeof(double) * nb, err);
  if (!err) err = make_schedule(P);
  if (!err) {
    size_t nl = 50 * (size_t)std::max<int64_t>(P.Lrmax, 1) * nb;
    P.evalv = (cd*)dalloc(P, sizeof(cd) * nl, err);
    P.etmp = (cd*)dalloc(P, sizeof(cd) * nl, err);
    P.ybuf = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.rbuf = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.xcore = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.dx = (cd*)dalloc(P, sizeof(cd) * (size_t)P.cn * nb, err);
    P.norms = (double*)dalloc(P, sizeof(double) * 4 * nb, err);
    size_t es = dtype == TIKH_C128 ? 16 : 8;
    P.d_in = dalloc(P, es * (size_t)(2 * m + 2 * n) + 64, err);
  }
  if (!err && cudaStreamSynchronize(P.stream) != cudaSuccess) err = TIKH_ECUDA;
  if (err) {
    cudaGetLastError();
    for (void* p : P.allocs) cudaFree(p);
    delete h;
    return err;
  }
  P.last.N = P.N;
  P.last.M = P.M;
  P.last.k = P.k;
  P.last.p = P.p;
  P.last.dual = P.dual;
  P.last.batch = 1;
  *out = h;
  return TIKH_OK;
}

int tikh_solve(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda)) return TIKH_EINVAL;
  return solve_with_retry(h->P, single(h->P, col, row, b, x), 0, &lambda, 1, nullptr, 0);
}

int tikh_solve_async(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda)) return TIKH_EINVAL;
  return enqueue_any(h->P, single(h->P, col, row, b, x), 0, &lambda, 1);
}

int tikh_solve_normal(tikh_plan h, const void* col, const void* row, const void* y, double lambda, void* x) {
  if (!h || !col || !row || !y || !x || !valid_lambda(lambda) || h->P.dual) return TIKH_EINVAL;
  return solve_with_retry(h->P, single(h->P, col, row, y, x), 1, &lambda, 1, nullptr, 0);
}

int tikh_solve_batched(tikh_plan h, int batch, const void* col, int64_t col_stride, const void* row,
                       int64_t row_stride, const void* b, int64_t b_stride, const double* lambdas, void* x,
                       int64_t x_stride) {
  if (!h || !col || !row || !b || !x || !lambdas || batch < 1 || batch > h->P.batch_max) return TIKH_EINVAL;
  if (col_stride < 0 || row_stride < 0 || b_stride < 0 || (batch > 1 && x_stride < h->P.n)) return TIKH_EINVAL;
  for (int i = 0; i < batch; ++i)
    if (!valid_lambda(lambdas[i])) return TIKH_EINVAL;
  UserArrays u;
  u.col = col;
  u.row = row;
  u.rhs = b;
  u.x = x;
  u.col_stride = col_stride;
  u.row_stride = row_stride;
  u.rhs_stride = b_stride;
  u.x_stride = x_stride;
  return solve_with_retry(h->P, u, 0, lambdas, batch, nullptr, 0);
}

int tikh_solve_grad(tikh_plan h, const void* col, const void* row, const void* b, double lambda, const void* x,
                    const void* dLdx, void* dLdcol, void* dLdrow, void* dLdb, double* dLdlambda) {
  if (!h || !col || !row || !b || !x || !dLdx || !dLdcol || !dLdrow || !dLdb || !dLdlambda || !valid_lambda(lambda))
    return TIKH_EINVAL;
  Plan& P = h->P;
  if (P.dual) return TIKH_EINVAL;  // the adjoint is implemented for m >= n
  int err = 0;
  if (!P.gbuf) {  // adjoint workspace, allocated by the first gradient call
    P.gbuf = (cd*)dalloc(P, sizeof(cd) * (size_t)(4 * P.N + 2 * P.cm) * (size_t)P.batch_max, err);
    P.gdl = (double*)dalloc(P, sizeof(double) * (size_t)P.batch_max, err);
    if (err) return err;
  }
  UserArrays u = single(P, col, row, dLdx, nullptr);
  int64_t nl = 0;
  int r;
  if ((r = enqueue_prologue(P, u, 1, &lambda, 1, nl)) < 0) return r;  // right-hand side y = dL/dx
  if ((r = enqueue_core_refined(P, nl)) < 0) return r;                // g = A^{-1} dL/dx
  if ((r = launch_grad(P, x, 0, b, 0, dLdcol, 0, dLdrow, 0, dLdb, 0, P.gdl, P.gbuf)) < 0) return r;
  nl += r;
  P.launches = nl;
  if (cudaMemcpyAsync(dLdlambda, P.gdl, sizeof(double), cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
    return TIKH_ECUDA;
  return sync_status(P);
}

int tikh_solve_host(tikh_plan h, const void* col, const void* row, const void* b, double lambda, void* x) {
  if (!h || !col || !row || !b || !x || !valid_lambda(lambda)) return TIKH_EINVAL;
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
  return solve_with_retry(P, single(P, dcol, drow, db, dx), 0, &lambda, 1, x, es * P.n);
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
  h->P.prof_leaf = flags & 3;
  h->P.ev_used = 0;
  h->P.last.prof_leaf_ms = 0.0;
  h->P.last.prof_leaf_launches = 0;
  for (int k = 0; k < 4; ++k) {
    h->P.last.prof_kind_ms[k] = 0.0;
    h->P.last.prof_kind_count[k] = 0;
  }
  return TIKH_OK;
}

void tikh_plan_destroy(tikh_plan h) {
  if (!h) return;
  cudaStreamSynchronize(h->P.stream);
  drop_graph(h->P);
  for (cudaEvent_t e : h->P.ev_pool) cudaEventDestroy(e);
  for (void* p : h->P.allocs) cudaFree(p);
  delete h;
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
