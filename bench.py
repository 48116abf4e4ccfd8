"""Benchmark: superfast Tikhonov solves of the deconvolution workload on GB300.

Workload (one step = one full solve: extension, transformation, recursive basis construction,
difficult points, extraction, optional refinement): complex128, m = 98304, n = 65536, Gaussian PSF
(sigma 8) with random phases, lambda = 1e-4.  value = solves/s over all ranks (weak scaling: every
rank solves its own problem).  Inputs are resident in HBM when the timed region starts; the working
set (~1 GB) exceeds L2 and L2 is also flushed between steps.  e2e repeats the measurement through
tikh_solve_host with host buffers (copies inside the timed region).

--impl reference times the CPU oracle (the paper's algorithm in plain C, FP64) on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s and n*solves/s at n=2^16..2^20 vs plain FP64 GPU at rel err<=1e-8; HBM %"

# FP64 peak of GB300 from its unit counts: 152 SMs x 4 sub-partitions x 0.5 DFMA/clk x 2 flop x clock
# (the sub-partition rate was measured: one FP64 warp instruction per 64 cycles).
FP64_PEAK_GFLOPS = 152 * 4 * 0.5 * 2 * 2.070


def leaf_model_flops(K):
    """Algorithmic FP64 flops of one leaf of K conditions (serial single-point construction):
    pivot chain sum_s [60 (K - s) + 60] (score 20 + update 40 per remaining condition, mu 60 per step)
    plus the basis rebuild ~20 K^2 (5 rows x ~K/10 coefficients x 40 flops per step)."""
    return 30 * K * K + 90 * K + 20 * K * K


# dram__bytes_read.sum + dram__bytes_write.sum of one k_leaf launch (K = 20, one problem), from
# profiles/k_leaf_c2recipe_n4096.md; None once the kernel changes after that capture
# dram__bytes_read.sum + dram__bytes_write.sum of one leaf launch (K = 20) from an ncu capture of the
# current kernel (profiles/k_leaf_c2recipe_n4096.md); None whenever the kernel changes until recaptured
LEAF_TRAFFIC_BYTES = 45056
# sm__inst_executed_pipe_fp64 (fraction of the SM's peak while the leaf runs) from the same capture
LEAF_FP64_PIPE_ACTIVE = 0.376


def model_bytes_per_solve(N, p):
    """Algorithmic HBM words of one solve (c128, 16 B each): per split level the left basis read
    for the evaluation (~5N), the right residuals read and written (~10N), both bases into the product
    (~10N) and the product out (~10N), about 35N; the leaves read their conditions and write their
    bases (~10N)."""
    return 16 * (35 * N * p + 10 * N)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed_offsets(rank, batch):
    """Weak scaling: rank r solves the problems with seed offsets r B .. r B + B - 1 (disjoint ranks)."""
    return [rank * batch + i for i in range(batch)]


def max_over_ranks(v, device=None):
    """The largest v over all ranks, returned on every rank (v itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, t_max_s):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / t_max_s


def workload(seed_offset=0, n=None):
    """c2: m = 98304, n = 65536; with n given, the same recipe at m = 1.5 n (the metric's n sweep)."""
    from paper_1302_6945_gb300 import workloads as W
    if n is None:
        return W.config_c2(seed=1 + seed_offset)
    return W.config_c2(seed=1 + seed_offset, m=3 * n // 2, n=n)


def run_reference(args, world, rank):
    """The CPU oracle on the host cores, on this arm's workload and metric."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    P = workload(n=args.n)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=args.n_lim)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    v = 1.0 / t
    out = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic", "impl": "reference",
           "config": {"workload": "deconvolution m=%d n=%d complex128 lambda=1e-4 (c2 recipe)" % (P["m"], P["n"]), "m": P["m"],
                      "n": P["n"], "n_lim": args.n_lim, "l2": "working set > L2"},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                            "sample": "full c2 solve per step, single thread"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-lim", type=int, default=32)
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="sweep point: n unknowns, m = 1.5 n (default: c2)")
    ap.add_argument("--batch", type=int, default=1, help="independent problems per step (tikh_solve_batched)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--prod-direct-max", type=int, default=0, help="direct products up to this P (0: automatic)")
    ap.add_argument("--eval-direct-max", type=int, default=0, help="direct evaluations up to this size (0: automatic)")
    ap.add_argument("--graph", type=int, default=1, help="1 (default): replay each solve as one captured CUDA graph; 0: stream launches")
    ap.add_argument("--single", action="store_true",
                    help="build the plan, run one solve of the workload and exit (a short command for profiler captures)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1302_6945_gb300 import tikh

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    B = max(1, args.batch)
    probs = [workload(seed_offset=o, n=args.n) for o in rank_seed_offsets(rank, B)]
    P = probs[0]
    m, n = P["m"], P["n"]
    col = torch.tensor(np.stack([q["col"] for q in probs]), dtype=torch.complex128, device=dev)
    row = torch.tensor(np.stack([q["row"] for q in probs]), dtype=torch.complex128, device=dev)
    bb = torch.tensor(np.stack([q["b"] for q in probs]), dtype=torch.complex128, device=dev)
    lams = [q["lam"] for q in probs]
    b = bb[0]
    xb = torch.empty((B, n), dtype=torch.complex128, device=dev)
    x = xb[0]
    stream = torch.cuda.Stream(device=dev)
    plan = tikh.Plan(m, n, "c128", n_lim=args.n_lim, refine_steps=args.refine, batch=B, graph=bool(args.graph),
                     prod_direct_max=args.prod_direct_max, eval_direct_max=args.eval_direct_max, stream=stream)

    def step(sync=True):
        if B == 1:
            plan.solve(col[0], row[0], bb[0], lams[0], x, sync=sync)
        else:
            plan.solve_batched(col, row, bb, lams, xb)
    if args.single:
        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize()
        st = plan.stats()
        print(json.dumps({"single_solve": True, "N": st["N"], "p": st["p"], "M": st["M"], "batch": B,
                          "kernel_launches": st["kernel_launches"]}))
        plan.close()
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    st = plan.stats()

    # accuracy of the benchmarked solution: relative residual of the normal equations (FFT matvec in
    # torch, outside the timed region)
    def normal_residual(xv):
        L = 1 << int(math.ceil(math.log2(m + 2 * n)))
        a = torch.cat([row[0, 1:].flip(0), col[0]])  # a_{-(n-1)} .. a_{m-1}
        A = torch.fft.fft(a, L)
        Tx = torch.fft.ifft(A * torch.fft.fft(xv, L))[n - 1:n - 1 + m]
        r = b - Tx
        # T^H r: correlate with conj(a)
        Ah = torch.fft.fft(a.conj().flip(0), L)
        Thr = torch.fft.ifft(Ah * torch.fft.fft(r, L))[m - 1:m - 1 + n]
        Thb = torch.fft.ifft(Ah * torch.fft.fft(b, L))[m - 1:m - 1 + n]
        return float(torch.linalg.norm(Thr - P["lam"] * xv) / torch.linalg.norm(Thb))

    res = normal_residual(x)

    # forward error of the benchmarked solution against a solve of the same problem with two FP64
    # refinement corrections (outside the timed region)
    ref_plan = tikh.Plan(m, n, "c128", n_lim=args.n_lim, refine_steps=max(2, args.refine + 1), stream=stream)
    with torch.cuda.stream(stream):
        x_ref = ref_plan.solve(col[0], row[0], bb[0], lams[0])
    ref_res = normal_residual(x_ref)
    rel_err_ref = float(torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
    ref_plan.close()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(sync=False)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    plan.sync()
    clocks = clk.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]

    # dominant kernel (the leaf): every launch timed with a CUDA event pair on the plan's stream, over
    # the same number of steps right after the timed region (events are not in the timed steps)
    plan.set_profiling(3)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            step(sync=True)
    plan.sync()
    pst = plan.stats()
    plan.set_profiling(0)
    kinds = ("leaf", "evaluation", "product", "other")
    breakdown = {k: {"ms_per_step": pst["prof_kind_ms"][i] / args.steps,
                     "groups_per_step": pst["prof_kind_count"][i] / args.steps} for i, k in enumerate(kinds)}
    t_step = sum(step_ms) / len(step_ms)
    t_max = max_over_ranks(t_step, dev)
    if world > 1:
        dist.barrier()
    value = whole_job_rate(world, B, t_max / 1e3)

    # e2e through the host-buffer entry point (pinned host arrays, copies inside the region)
    hcol = torch.tensor(P["col"], dtype=torch.complex128).pin_memory().numpy()
    hrow = torch.tensor(P["row"], dtype=torch.complex128).pin_memory().numpy()
    hb = torch.tensor(P["b"], dtype=torch.complex128).pin_memory().numpy()
    hx = torch.empty(n, dtype=torch.complex128).pin_memory().numpy()
    e2e_t = float("nan")
    if not args.no_e2e:
        plan.solve_host(hcol, hrow, hb, P["lam"], hx)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.solve_host(hcol, hrow, hb, P["lam"], hx)
        e2e_t = (time.perf_counter() - t0) / args.steps
    e2e_v = 1.0 / e2e_t  # host-buffer path solves one problem per call
    if world > 1 and not args.no_e2e:
        e2e_v = whole_job_rate(world, 1, max_over_ranks(e2e_t, dev))

    pk, pk_kind = peaks()
    K_leaf = 2 * int(st["M"])
    leaf_launches = max(1, int(pst["prof_leaf_launches"]))
    leaf_ms = max(pst["prof_leaf_ms"] / leaf_launches, 1e-9)
    leaf_gflops = leaf_model_flops(K_leaf) * B / (leaf_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "kernel": "k_leaf (FP64 serial single-point construction)",
                "achieved": leaf_gflops, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": leaf_gflops / FP64_PEAK_GFLOPS, "peak_kind": "derived from unit counts and max clock",
                "traffic": LEAF_TRAFFIC_BYTES, "avg_launch_ms": leaf_ms,
                # a leaf is one CTA: a single solve can use one SM's FP64 units at most
                "peak_one_sm": FP64_PEAK_GFLOPS / 152, "frac_of_one_sm": leaf_gflops / B / (FP64_PEAK_GFLOPS / 152),
                "fp64_pipe_active_ncu": LEAF_FP64_PIPE_ACTIVE,
                "launches_per_step": leaf_launches / args.steps,
                "share_of_step": (pst["prof_leaf_ms"] / args.steps) / t_step,
                "flops_per_launch": leaf_model_flops(K_leaf) * B}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        xo, _ = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=args.n_lim)
        tc = time.perf_counter() - t0
        err = float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo))
        cpu = {"value": 1.0 / tc, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "one full solve of the same problem (m=%d, n=%d), single thread" % (m, n), "gpu_vs_oracle_rel_err": err}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "c128", "data": "synthetic",
               "config": {"workload": "deconvolution m=%d n=%d complex128 lambda=1e-4 (c2 recipe)" % (m, n), "m": m, "n": n,
                          "N": st["N"], "p": st["p"], "M": st["M"], "n_lim": args.n_lim,
                          "refine_steps": args.refine, "precision": "fp64", "batch": B,
                          "cuda_graph": bool(st["graph"]),
                          "prod_direct_max": args.prod_direct_max or "auto", "eval_direct_max": args.eval_direct_max or "auto",
                          "l2": "256 MB flush between steps; working set > L2"},
               "n_solves_per_s": value * n,
               "solves_per_s_per_problem_stream": value / B,
               "normal_eq_rel_residual": res,
               "rel_err_vs_refined": {"value": rel_err_ref, "reference": "same problem, %d FP64 refinement "
                                      "corrections" % max(2, args.refine + 1), "reference_normal_eq_rel_residual":
                                      ref_res},
               "e2e": {"value": e2e_v, "unit": "solves/s", "h2d_bytes_per_step": 16 * (2 * m + n),
                       "d2h_bytes_per_step": 16 * n},
               "gpu_launches": int(st["kernel_launches"]) * args.steps,
               "clocks": clocks,
               "peaks": {"hbm_gbs": pk.get("hbm_gbs"), "kind": pk_kind},
               "roofline": roofline,
               "hbm": {"model_bytes_per_solve": model_bytes_per_solve(st["N"], st["p"]),
                       "achieved_gbs": model_bytes_per_solve(st["N"], st["p"]) * B / (t_max / 1e3) / 1e9,
                       "pct_of_measured": 100.0 * model_bytes_per_solve(st["N"], st["p"]) * B / (t_max / 1e3) / 1e9
                       / pk.get("hbm_gbs", 6788.3)},
               "step_breakdown": breakdown,
               "cpu_baseline": cpu}
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
