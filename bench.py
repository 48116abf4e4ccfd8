"""Benchmark: superfast Tikhonov solves of the deconvolution workload on GB300.

Default workload (one step = one full solve: extension, transformation, recursive basis construction,
difficult points, extraction, optional refinement): complex128, m = 98304, n = 65536, Gaussian PSF
(sigma 8) with random phases, lambda = 1e-4 (plain FP64).  value = solves/s over all ranks (weak scaling:
every rank solves its own problem).  Inputs are resident in HBM when the timed region starts; the working
set (~1 GB) exceeds L2 and L2 is also flushed between steps.  e2e repeats the measurement through
tikh_solve_host with host buffers (copies inside the timed region).  The default run also reports the
metric's n sweep (n = 2^17 .. 2^20, m = 1.5 n, one FP64 refinement correction) under "sweep".
The same run times one solve of the general problem (Sec. 3.2, T and L 65536 x 65536) under
"general_problem", and under "many_rhs" the benchmarked T and lambda with 16 right-hand sides per call
through the displacement representation of the inverse (tikh_inverse_*, an extension of the paper).

--config c3 runs the batching configuration instead: 512 real problems of uneven shape, each with a
16-value regularisation path, as one ragged batch (tikh_solve_batched, one captured graph per call).
--config general runs the general problem (Sec. 3.2) with square T and L as the main line.
--precision selects FP64, FP32 stages, or FP32 stages with FP64 refinement.
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
KINDS = ("leaf", "evaluation", "product", "other")

# dram__bytes_read.sum + dram__bytes_write.sum of one leaf launch (K = 20, one problem): the mean of two
# launches of an ncu capture with warm caches (--cache-control none) of the current leaf kernel at n = 4096
# (the same K = 20 kernel as the c2 workload); None whenever the kernel changes until it is recaptured
LEAF_TRAFFIC_BYTES = 640
LEAF_TRAFFIC_NOTE = "ncu, warm caches, c2 recipe at n = 4096 (same K = 20 kernel), mean of 2 launches"


def model_bytes_per_solve(N, p, word=16):
    """Algorithmic HBM bytes of one core solve: per split level the left basis read for the evaluation
    (~5N words), the right residuals read and written (~10N), both bases into the product (~10N) and the
    product out (~10N), about 35N; the leaves read their conditions and write their bases (~10N)."""
    return word * (35 * N * p + 10 * N)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fma_peaks(tikh, stream):
    """Measured FP64 and FP32 FMA rates of this GPU (GFLOP/s), by the library's peak-rate kernel."""
    return tikh.tikh_test_peak(0, stream), tikh.tikh_test_peak(1, stream)


def kind_rooflines(st, pst, steps, items, solves_per_item, p64, p32):
    """Per kind of launch group (leaf, evaluation, product, other): model FLOPs of the groups (the library's
    algorithmic count per core solve x items x core solves per item) over their event-timed duration, as a
    fraction of the measured FMA peak of the precision they run in (FP32 for the FP32-stage share)."""
    out = {}
    for i, k in enumerate(KINDS):
        t = pst["prof_kind_ms"][i] / steps * 1e-3
        f = st["model_flops"][i] * items * solves_per_item
        f32 = st["model_flops_fp32"][i] * items * solves_per_item
        if t <= 0:
            continue
        # the time the kind's flops need at the two peaks, over the time it took
        t_peak = (f - f32) / (p64 * 1e9) + f32 / (p32 * 1e9)
        out[k] = {"ms_per_step": t * 1e3, "model_gflop_per_step": f / 1e9, "fp32_share_of_flops": f32 / f if f else 0.0,
                  "achieved_gflops": f / t / 1e9, "frac_of_peak": t_peak / t,
                  "groups_per_step": pst["prof_kind_count"][i] / steps}
    return out


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


def c3_reference_sample(count=8, seed=11):
    """A bounded, seeded sample of the batching configuration's items (problem, lambda): `count` items drawn
    uniformly from the 512 x 16, so the mean time per item estimates the whole workload's."""
    import numpy as np
    from paper_1302_6945_gb300 import workloads as W
    probs, lams = W.batch_c3()
    rng = np.random.default_rng(seed)
    ids = rng.choice(len(probs) * len(lams), size=count, replace=False)
    return [(probs[i // len(lams)], float(lams[i % len(lams)])) for i in sorted(ids)], len(probs) * len(lams)


def _oracle_item(item):
    """One oracle solve of a batch item (a pool worker; the oracle is single-threaded); its time in s."""
    import oracle
    col, row, b, lam, n_lim = item
    t0 = time.perf_counter()
    oracle.solve(col, row, b, lam, nlim=n_lim, is_complex=0)
    return time.perf_counter() - t0


def c3_oracle_all_cores(n_lim, per_core=2, seed=11):
    """The oracle on every host core, one item (problem, lambda) per process at a time: a bounded sample of
    per_core x cores items of the batching configuration drawn uniformly; items / wall time (the slowest
    items finish last, so this is below cores x the one-core rate)."""
    import multiprocessing
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    sample, total = c3_reference_sample(count=min(per_core * cores, 8192), seed=seed)
    items = [(P["col"], P["row"], P["b"], lam, n_lim) for P, lam in sample]
    ctx = multiprocessing.get_context("spawn")  # safe after the process has used the GPU
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_item, [(P["col"][:64], P["row"][:64], P["b"][:64], lam, n_lim)
                                for P, lam in sample[:cores]])  # workers up, oracle loaded
        t0 = time.perf_counter()
        per_item = pool.map(_oracle_item, sorted(items, key=lambda it: -len(it[0])), chunksize=1)
        t = time.perf_counter() - t0
    return {"value": len(items) / t, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "cpu_seconds": sum(per_item), "wall_seconds": t,
            "sample": "%d items (problem, lambda) drawn uniformly from the %d, one process per core, largest "
                      "first" % (len(items), total)}


def run_reference(args, world, rank):
    """The CPU oracle on the host cores, on this arm's workload and metric."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    if args.config == "c3":
        sample, total = c3_reference_sample()
        times = []
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            for P, lam in sample:
                oracle.solve(P["col"], P["row"], P["b"], lam, nlim=args.n_lim, is_complex=0)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
        t = sum(times) / len(times)
        v = len(sample) / t
        allc = c3_oracle_all_cores(args.n_lim)
        cfg = {"workload": "c3: 512 real deconvolution problems, n log-uniform in [256, 65536], m = n + U[0, n/2], "
                           "16-value lambda path 1e-6..1 (8192 solves)", "n_lim": args.n_lim,
               "all_cores": allc}
        out = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference", "config": cfg,
               "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                "sample": "%d items (problem, lambda) drawn uniformly from the %d, single thread, "
                                          "each solved plainly" % (len(sample), total)},
               "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
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
           "config": {"workload": "deconvolution m=%d n=%d complex128 lambda=1e-4 (c2 recipe)" % (P["m"], P["n"]),
                      "m": P["m"], "n": P["n"], "n_lim": args.n_lim, "l2": "working set > L2"},
           "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                            "sample": "full c2 solve per step, single thread"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def normal_residual_t(torch, col, row, b, xv, lam):
    """||T^H (b - T x) - lam x|| / ||T^H b|| by FFT convolutions in torch (outside any timed region)."""
    col, row, b, xv = (v.to(torch.complex128) for v in (col, row, b, xv))
    m, n = col.numel(), row.numel()
    L = 1 << int(math.ceil(math.log2(m + 2 * n)))
    a = torch.cat([row[1:].flip(0), col])  # a_{-(n-1)} .. a_{m-1}
    A = torch.fft.fft(a, L)
    Ah = torch.fft.fft(a.conj().flip(0), L)
    Tx = torch.fft.ifft(A * torch.fft.fft(xv, L))[n - 1:n - 1 + m]
    Thr = torch.fft.ifft(Ah * torch.fft.fft(b - Tx, L))[m - 1:m - 1 + n]
    Thb = torch.fft.ifft(Ah * torch.fft.fft(b, L))[m - 1:m - 1 + n]
    return float(torch.linalg.norm(Thr - lam * xv) / torch.linalg.norm(Thb))


def toeplitz_mv_t(torch, col, row, v, adjoint=False):
    """T v (or T^H v) for the Toeplitz T = [col, row] by one FFT convolution in torch."""
    m, n = col.numel(), row.numel()
    L = 1 << int(math.ceil(math.log2(m + n)))
    a = torch.cat([row[1:].flip(0), col])  # a_{-(n-1)} .. a_{m-1}
    if not adjoint:
        return torch.fft.ifft(torch.fft.fft(a, L) * torch.fft.fft(v, L))[n - 1:n - 1 + m]
    return torch.fft.ifft(torch.fft.fft(a.conj().flip(0), L) * torch.fft.fft(v, L))[m - 1:m - 1 + n]


def general_residual_t(torch, col, row, lcol, lrow, b, xv):
    """||T^H b - (T^H T + L^H L) x|| / ||T^H b|| (outside any timed region)."""
    col, row, lcol, lrow, b, xv = (v.to(torch.complex128) for v in (col, row, lcol, lrow, b, xv))
    y = toeplitz_mv_t(torch, col, row, b, True)
    ax = toeplitz_mv_t(torch, col, row, toeplitz_mv_t(torch, col, row, xv), True) + \
        toeplitz_mv_t(torch, lcol, lrow, toeplitz_mv_t(torch, lcol, lrow, xv), True)
    return float(torch.linalg.norm(y - ax) / torch.linalg.norm(y))


def run_general(args, world, rank, local):
    """The general problem (Sec. 3.2) on its own line: square T and L (m = p = n, the paper's Sec. 7.1 case)
    with standard-normal generators, one solve per step (weak scaling: rank r solves its own problem,
    seed 20 + r)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1302_6945_gb300 import tikh
    from paper_1302_6945_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = args.n or 65536
    P = W.general_problem(n, n, n, seed=20 + rank)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    col, row, lcol, lrow, b = t(P["col"]), t(P["row"]), t(P["lcol"]), t(P["lrow"]), t(P["b"])
    x = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    plan = tikh.GeneralPlan(n, n, n, "r64", n_lim=args.n_lim, refine_steps=args.refine, graph=bool(args.graph),
                            stream=stream)
    if args.single:
        with torch.cuda.stream(stream):
            plan.solve(col, row, lcol, lrow, b, x)
        torch.cuda.synchronize()
        st = plan.stats()
        print(json.dumps({"single_solve": True, "general": True, "N": st["N"], "p": st["p"], "M": st["M"],
                          "kernel_launches": st["kernel_launches"]}))
        plan.close()
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.solve(col, row, lcol, lrow, b, x)
    st = plan.stats()
    rel_res = general_residual_t(torch, col, row, lcol, lrow, b, x)
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
            plan.solve(col, row, lcol, lrow, b, x)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_step = sum(a.elapsed_time(c) for a, c in ev) / args.steps
    t_max = max_over_ranks(t_step, dev)
    value = whole_job_rate(world, 1, t_max / 1e3)
    # profiled pass: every launch group timed by kind (stream launches)
    plan.set_profiling(3)
    with torch.cuda.stream(stream):
        plan.solve(col, row, lcol, lrow, b, x)
    torch.cuda.synchronize()
    pst = plan.stats()
    plan.set_profiling(0)
    # e2e: the problem in pinned host memory, copies in and the solution out inside the timed region
    host = [torch.tensor(P[k], dtype=torch.float64).pin_memory() for k in ("col", "row", "lcol", "lrow", "b")]
    hx = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    with torch.cuda.stream(stream):
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for dst, src in zip((col, row, lcol, lrow, b), host):
                dst.copy_(src, non_blocking=True)
            plan.solve(col, row, lcol, lrow, b, x)
            hx.copy_(x, non_blocking=True)
            stream.synchronize()
            e2e_times.append(time.perf_counter() - t0)
    e2e_v = whole_job_rate(world, 1, max_over_ranks(sum(e2e_times) / len(e2e_times), dev))
    h2d = sum(8 * h.numel() for h in host)
    p64, p32 = fma_peaks(tikh, stream.cuda_stream)
    solves = 1 + args.refine
    kr = kind_rooflines(st, pst, 1, 1, solves, p64, p32)
    dom = max(kr, key=lambda k: kr[k]["ms_per_step"]) if kr else None
    roof = None
    if dom:
        d = kr[dom]
        roof = {"bound": "alu", "kernel": "%s launch groups (profiled pass)" % dom, "achieved": d["achieved_gflops"],
                "unit": "GFLOP/s", "peak": p64, "peak_kind": "measured FP64 FMA rate (tikh_test_peak)",
                "frac": d["frac_of_peak"],
                "frac_note": "time the group's model FLOPs need at the measured FP64 peak over its time",
                "traffic": None}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        y = toeplitz_mv_t(torch, col.cpu().to(torch.complex128), row.cpu().to(torch.complex128),
                          b.cpu().to(torch.complex128), True).numpy()
        t0 = time.perf_counter()
        xo, _ = oracle.solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=args.n_lim, is_complex=0)
        dt = time.perf_counter() - t0
        xg = x.cpu().numpy()
        cpu = {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "one full solve of the same problem, single thread",
               "rel_diff_gpu_vs_oracle": float(np.linalg.norm(xg - xo.real) / np.linalg.norm(xo.real))}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": "general problem (Sec. 3.2): min ||T x - b||^2 + ||L x||^2, T and L %d x %d "
                                      "real Toeplitz with standard-normal generators, b = T x_true" % (n, n),
                          "m": n, "n": n, "pl": n, "N": st["N"], "p": st["p"], "M": st["M"], "n_lim": args.n_lim,
                          "refine_steps": args.refine, "cuda_graph": bool(st["graph"]),
                          "l2": "256 MB flush between steps"},
               "accuracy": {"rel_residual": rel_res, "n_difficult": st["n_difficult"]},
               "e2e": {"value": e2e_v, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * n},
               "gpu_launches": int(st["kernel_launches"]) * args.steps, "clocks": clocks,
               "fma_peaks_gflops": {"fp64": p64, "fp32": p32}, "roofline": roof, "kinds": kr, "cpu_baseline": cpu}
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_c3(args, world, rank, local):
    """The batching configuration as one ragged batch per step (weak scaling: rank r solves its own
    512-problem set, seed 2 + r)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1302_6945_gb300 import tikh
    from paper_1302_6945_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    probs, lams = W.batch_c3(seed=2 + rank)
    L = len(lams)
    ms, ns = [p["m"] for p in probs], [p["n"] for p in probs]
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    cols, rows, bs = [t(p["col"]) for p in probs], [t(p["row"]) for p in probs], [t(p["b"]) for p in probs]
    xs = [torch.empty(n, dtype=torch.float64, device=dev) for n in ns for _ in range(L)]
    stream = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    bp = tikh.BatchPlan(ms, ns, L, "r64", n_lim=args.n_lim, refine_steps=args.refine, graph=bool(args.graph),
                        precision=args.precision, stream=stream)
    t_plan = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            bp.solve(cols, rows, bs, lams, xs)
    st = bp.stats()
    # accuracy on a sample of items against single FP64 solves with two refinement corrections
    rng = np.random.default_rng(7)
    pick = sorted(rng.choice(len(probs), size=6, replace=False).tolist()) + [int(np.argmax(ns))]
    errs = []
    with torch.cuda.stream(stream):
        for i in pick:
            l = int(rng.integers(L))
            ref = tikh.Plan(ms[i], ns[i], "r64", n_lim=args.n_lim, refine_steps=2, stream=stream)
            xr = ref.solve(cols[i], rows[i], bs[i], float(lams[l]))
            ref.close()
            x = xs[i * L + l]
            errs.append(float(torch.linalg.norm(x - xr) / torch.linalg.norm(xr)))
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
            bp.solve(cols, rows, bs, lams, xs)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_step = sum(step_ms) / len(step_ms)
    t_max = max_over_ranks(t_step, dev)
    items = len(probs) * L
    value = whole_job_rate(world, items, t_max / 1e3)
    # profiled pass (groups one after another, every launch group timed by kind)
    bp.set_profiling(2)
    with torch.cuda.stream(stream):
        bp.solve(cols, rows, bs, lams, xs)
    torch.cuda.synchronize()
    pst = bp.stats()
    bp.set_profiling(0)
    # e2e: the same call with the problems in pinned host memory, copies inside the timed region
    hc = [torch.tensor(p["col"], dtype=torch.float64).pin_memory() for p in probs]
    hr = [torch.tensor(p["row"], dtype=torch.float64).pin_memory() for p in probs]
    hb = [torch.tensor(p["b"], dtype=torch.float64).pin_memory() for p in probs]
    hx = [torch.empty(n, dtype=torch.float64).pin_memory() for n in ns for _ in range(L)]
    h2d = sum(8 * (a.numel() + b.numel() + c.numel()) for a, b, c in zip(hc, hr, hb))
    d2h = sum(8 * x.numel() for x in hx)
    e2e_times = []
    with torch.cuda.stream(stream):
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for dst, src in zip(cols + rows + bs, hc + hr + hb):
                dst.copy_(src, non_blocking=True)
            bp.solve(cols, rows, bs, lams, xs)
            for dst, src in zip(hx, xs):
                dst.copy_(src, non_blocking=True)
            stream.synchronize()
            e2e_times.append(time.perf_counter() - t0)
    e2e_t = sum(e2e_times) / len(e2e_times)
    e2e_v = whole_job_rate(world, items, max_over_ranks(e2e_t, dev))
    p64, p32 = fma_peaks(tikh, stream.cuda_stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = c3_oracle_all_cores(args.n_lim)
    nref = args.refine if args.refine > 0 else (2 if args.precision == "fp32_refine" else 0)
    solves = 1 + nref
    pst_one = dict(pst)
    kr = kind_rooflines({"model_flops": [f / items for f in pst["model_flops"]],
                         "model_flops_fp32": [f / items for f in pst["model_flops_fp32"]]},
                        pst_one, 1, items, solves, p64, p32)
    dom = max(kr, key=lambda k: kr[k]["ms_per_step"]) if kr else None
    roof = None
    if dom:
        d = kr[dom]
        f32 = d["fp32_share_of_flops"]
        roof = {"bound": "alu", "kernel": "%s launch groups of the ragged batch (profiled pass, groups serialised)" % dom,
                "achieved": d["achieved_gflops"], "unit": "GFLOP/s",
                "peak": p64 if f32 < 0.5 else p32, "peak_kind": "measured FMA rate (tikh_test_peak), %s"
                % ("FP64" if f32 < 0.5 else "FP32"), "frac": d["frac_of_peak"],
                "frac_note": "time the group's model FLOPs need at the measured FP64/FP32 peaks over its time",
                "traffic": None}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 stages + f64",
               "data": "synthetic",
               "config": {"workload": "c3: 512 real deconvolution problems, n log-uniform in [256, 65536], "
                                      "m = n + U[0, n/2], sigma ~ U[2, 16], 16-value lambda path 1e-6..1 "
                                      "(8192 solves per step, one ragged batch)",
                          "items": items, "precision": args.precision, "refine_steps": solves - 1,
                          "groups": st["ngroups"], "max_waves": st["max_waves"], "cuda_graph": bool(st["graph"]),
                          "workspace_bytes": st["workspace_bytes"], "plan_s": t_plan,
                          "l2": "256 MB flush between steps; working set > L2"},
               "accuracy": {"sampled_items": len(errs), "max_rel_err_vs_fp64_refined": max(errs),
                            "reference": "single FP64 solves with 2 refinement corrections",
                            "max_rel_residual": st["rel_residual"]},
               "e2e": {"value": e2e_v, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": int(st["kernel_launches"]) * args.steps, "clocks": clocks,
               "fma_peaks_gflops": {"fp64": p64, "fp32": p32}, "roofline": roof, "kinds": kr,
               "cpu_baseline": cpu}
        print(json.dumps(out))
    bp.close()
    if world > 1:
        dist.destroy_process_group()


def sweep_point(tikh, torch, n, refine, args, stream, dev):
    """One point of the metric's sweep: the c2 recipe at n, m = 1.5 n, `refine` FP64 corrections; one warm-up
    (graph capture) and args.sweep_steps timed solves."""
    P = workload(n=n)
    m = P["m"]
    t = lambda a: torch.tensor(a, dtype=torch.complex128, device=dev)
    col, row, b = t(P["col"]), t(P["row"]), t(P["b"])
    x = torch.empty(n, dtype=torch.complex128, device=dev)
    plan = tikh.Plan(m, n, "c128", n_lim=args.n_lim, refine_steps=refine, graph=True, stream=stream)
    with torch.cuda.stream(stream):
        plan.solve(col, row, b, P["lam"], x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sweep_steps):
            plan.solve(col, row, b, P["lam"], x, sync=False)
        e1.record(stream)
        e1.synchronize()
        plan.sync()
    st = plan.stats()
    ms = e0.elapsed_time(e1) / args.sweep_steps
    res = normal_residual_t(torch, col, row, b, x, P["lam"])
    plan.close()
    return {"n": n, "m": m, "N": st["N"], "refine_steps": refine, "ms_per_solve": ms, "solves_per_s": 1e3 / ms,
            "n_solves_per_s": n * 1e3 / ms, "normal_eq_rel_residual": res,
            "library_rel_residual": st["rel_residual"],
            "last_correction_rel": st["last_correction"],
            "accuracy_note": "last_correction_rel = ||dx||/||x|| of the last correction, the error of the solution "
                             "before it; each FP64 correction contracts the error (measured: <= 1.4e-11 after one "
                             "correction at n = 2^20 against two)"}


def many_rhs_point(tikh, torch, P, col, row, x_ref, superfast_ms, p64, args, stream, dev, R=16):
    """Many right-hand sides of the benchmarked T and lambda (tikh_inverse_*, an extension of the paper): the
    displacement representation of (T^H T + lam I)^{-1} from eight superfast solves (one batch of 8, one FP64
    correction each), then R right-hand sides per apply (T^H b, ten transforms, one correction of fourteen).
    Right-hand side 0 is the benchmarked b, whose solution is compared with the refined superfast solve."""
    import numpy as np
    m, n, lam = P["m"], P["n"], P["lam"]
    rng = np.random.default_rng(31)
    bs = np.stack([P["b"]] + [P["b"] + 0.05 * np.abs(P["b"]).max() * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
                              for _ in range(R - 1)])
    bt = torch.tensor(bs, dtype=torch.complex128, device=dev)
    xs = torch.empty((R, n), dtype=torch.complex128, device=dev)
    plan = tikh.Plan(m, n, "c128", n_lim=args.n_lim, refine_steps=1, batch=8, graph=True, stream=stream)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inv = tikh.Inverse(plan, col, row, lam, max_rhs=R)
        create_ms = (time.perf_counter() - t0) * 1e3
        create_launches = inv.info()["kernel_launches"]
        inv.apply(bt, refine_steps=1, x=xs)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(3, args.sweep_steps)
        e0.record(stream)
        for _ in range(steps):
            inv.apply(bt, refine_steps=1, x=xs)
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    info = inv.info()
    N = plan.stats()["N"]
    err = float(torch.linalg.norm(xs[0] - x_ref) / torch.linalg.norm(x_ref))
    inv.close()
    plan.close()
    transforms = R * (12 + 14)  # from b: T^H b and the apply; one correction
    flops = transforms * 5.0 * N * math.log2(N)
    per_rhs = ms / R
    return {"what": "many right-hand sides of one T and lambda: displacement representation of (T^H T + lam I)^-1 "
                    "(eight superfast solves), then FFT applies (tikh_inverse_create / tikh_inverse_apply)",
            "rhs_per_apply": R, "ms_per_apply": ms, "rhs_per_s": R * 1e3 / ms, "ms_per_rhs": per_rhs,
            "create_ms": create_ms, "create_kernel_launches": create_launches,
            "apply_kernel_launches": info["kernel_launches"], "workspace_bytes": info["workspace_bytes"],
            "superfast_ms_per_solve": superfast_ms,
            "speedup_per_extra_rhs": superfast_ms / per_rhs,
            "break_even_rhs": create_ms / max(superfast_ms - per_rhs, 1e-9),
            "rel_err_vs_refined_superfast": err, "refine_steps": 1,
            "fft_fp64": {"model_flops_per_apply": flops, "model": "5 N log2 N per length-N transform, %d transforms"
                         % transforms, "achieved_gflops": flops / (ms * 1e-3) / 1e9,
                         "frac_of_fp64_peak": flops / (ms * 1e-3) / 1e9 / p64}}


def general_point(tikh, torch, n, args, stream, dev):
    """The general problem (Sec. 3.2) at T, L n x n: one warm-up (graph capture) and args.sweep_steps timed
    solves, the normal-equation residual of the result."""
    from paper_1302_6945_gb300 import workloads as W
    P = W.general_problem(n, n, n, seed=20)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    col, row, lcol, lrow, b = t(P["col"]), t(P["row"]), t(P["lcol"]), t(P["lrow"]), t(P["b"])
    x = torch.empty(n, dtype=torch.float64, device=dev)
    plan = tikh.GeneralPlan(n, n, n, "r64", graph=True, stream=stream)
    with torch.cuda.stream(stream):
        plan.solve(col, row, lcol, lrow, b, x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sweep_steps):
            plan.solve(col, row, lcol, lrow, b, x)
        e1.record(stream)
        e1.synchronize()
    st = plan.stats()
    ms = e0.elapsed_time(e1) / args.sweep_steps
    res = general_residual_t(torch, col, row, lcol, lrow, b, x)
    plan.close()
    return {"problem": "general (Sec. 3.2): T and L %d x %d real Toeplitz, standard-normal generators" % (n, n),
            "N": st["N"], "M": st["M"], "ms_per_solve": ms, "solves_per_s": 1e3 / ms,
            "normal_eq_rel_residual": res, "n_difficult": st["n_difficult"],
            "full_line": "bench.py --config general"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "general"],
                    help="c2 (default): the complex deconvolution solve; c3: the ragged batch of 512 problems x 16 "
                         "lambdas; general: the general problem (Sec. 3.2) with square T and L (--n, default 65536)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32_refine"])
    ap.add_argument("--n-lim", type=int, default=None,
                    help="leaf size limit N_lim (conditions per leaf): default 32, or 30 for --config general")
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="sweep point: n unknowns, m = 1.5 n (default: c2)")
    ap.add_argument("--batch", type=int, default=1, help="independent problems per step (tikh_solve_strided)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n = 2^17 .. 2^20 sweep of the default run")
    ap.add_argument("--sweep-steps", type=int, default=1)
    ap.add_argument("--prod-direct-max", type=int, default=0, help="direct products up to this P (0: automatic)")
    ap.add_argument("--eval-direct-max", type=int, default=0, help="direct evaluations up to this size (0: automatic)")
    ap.add_argument("--graph", type=int, default=1, help="1 (default): replay each solve as one captured CUDA graph; 0: stream launches")
    ap.add_argument("--single", action="store_true",
                    help="build the plan, run one solve of the workload and exit (a short command for profiler captures)")
    args = ap.parse_args()
    if args.n_lim is None:
        args.n_lim = 30 if args.config == "general" else 32
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.config == "c3":
        return run_c3(args, world, rank, local)
    if args.config == "general":
        return run_general(args, world, rank, local)

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
                     prod_direct_max=args.prod_direct_max, eval_direct_max=args.eval_direct_max,
                     precision=args.precision, stream=stream)

    def step(sync=True):
        if B == 1:
            plan.solve(col[0], row[0], bb[0], lams[0], x, sync=sync)
        else:
            plan.solve_strided(col, row, bb, lams, xb)
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
    res = normal_residual_t(torch, col[0], row[0], b, x, P["lam"])

    # forward error of the benchmarked solution against a solve of the same problem with two FP64
    # refinement corrections (outside the timed region)
    nref = max(2, args.refine + 1)
    ref_plan = tikh.Plan(m, n, "c128", n_lim=args.n_lim, refine_steps=nref, stream=stream)
    with torch.cuda.stream(stream):
        x_ref = ref_plan.solve(col[0], row[0], bb[0], lams[0])
    ref_res = normal_residual_t(torch, col[0], row[0], b, x_ref, P["lam"])
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

    # every launch group timed with a CUDA event pair on the plan's stream, over the same number of
    # steps right after the timed region (events are not in the timed steps)
    plan.set_profiling(3)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            step(sync=True)
    plan.sync()
    pst = plan.stats()
    plan.set_profiling(0)
    breakdown = {k: {"ms_per_step": pst["prof_kind_ms"][i] / args.steps,
                     "groups_per_step": pst["prof_kind_count"][i] / args.steps} for i, k in enumerate(KINDS)}
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
    p64, p32 = fma_peaks(tikh, stream.cuda_stream)
    solves_per_item = 1 + int(st["refine_steps"])
    kr = kind_rooflines(st, pst, args.steps, B, solves_per_item, p64, p32)
    dom = max(kr, key=lambda k: kr[k]["ms_per_step"])
    if dom == "leaf":
        # the leaf as one kernel: model FLOPs per launch over its event-timed average launch duration
        leaf_launches = max(1, int(pst["prof_leaf_launches"]))
        leaf_ms = max(pst["prof_leaf_ms"] / leaf_launches, 1e-9)
        leaves = 1 << int(st["p"])
        flops_launch = st["model_flops"][0] / leaves * B
        ach = flops_launch / (leaf_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "kernel": "k_leaf (FP64 serial single-point construction)",
                    "achieved": ach, "peak": p64, "unit": "GFLOP/s", "frac": ach / p64,
                    "peak_kind": "measured FP64 FMA rate of this GPU (tikh_test_peak)",
                    "traffic": LEAF_TRAFFIC_BYTES if B == 1 else None, "traffic_note": LEAF_TRAFFIC_NOTE,
                    "avg_launch_ms": leaf_ms, "flops_per_launch": flops_launch,
                    # a leaf is one CTA: a single solve can use one SM's FP64 units at most
                    "peak_one_sm": p64 / 152, "frac_of_one_sm": ach / B / (p64 / 152),
                    "launches_per_step": leaf_launches / args.steps,
                    "share_of_step": (pst["prof_leaf_ms"] / args.steps) / t_step}
    else:
        d = kr[dom]
        f32 = d["fp32_share_of_flops"]
        roofline = {"bound": "alu", "kernel": "%s launch groups (FFT tiles and their pointwise kernels)" % dom,
                    "achieved": d["achieved_gflops"], "unit": "GFLOP/s", "peak": p64 if f32 < 0.5 else p32,
                    "peak_kind": "measured %s FMA rate of this GPU (tikh_test_peak)" % ("FP64" if f32 < 0.5 else "FP32"),
                    "frac": d["frac_of_peak"],
                    "frac_note": "time the groups' model FLOPs need at the measured FP64/FP32 peaks over their time",
                    "traffic": None, "share_of_step": d["ms_per_step"] / t_step}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        xo, _ = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=args.n_lim)
        tc = time.perf_counter() - t0
        xr = x_ref.cpu().numpy()
        err = float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo))
        cpu = {"value": 1.0 / tc, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "one full solve of the same problem (m=%d, n=%d), single thread" % (m, n),
               "gpu_vs_oracle_rel_err": err,
               "oracle_vs_refined_rel_err": float(np.linalg.norm(xo - xr) / np.linalg.norm(xr)),
               "gpu_vs_refined_rel_err": rel_err_ref}

    sweep = None
    if rank == 0 and world == 1 and not args.no_sweep and args.n is None and B == 1 and args.precision == "fp64":
        sweep = []
        for e in range(17, 21):
            sweep.append(sweep_point(tikh, torch, 1 << e, 1, args, stream, dev))
    general = None
    if rank == 0 and world == 1 and not args.no_sweep and args.n is None and B == 1 and args.precision == "fp64":
        general = general_point(tikh, torch, 1 << 16, args, stream, dev)
    many = None
    if rank == 0 and world == 1 and not args.no_sweep and args.n is None and B == 1 and args.precision == "fp64":
        many = many_rhs_point(tikh, torch, P, col[0], row[0], x_ref, t_step, p64, args, stream, dev)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else "c64 stages + c128",
               "data": "synthetic",
               "config": {"workload": "deconvolution m=%d n=%d complex128 lambda=1e-4 (c2 recipe)" % (m, n),
                          "m": m, "n": n, "N": st["N"], "p": st["p"], "M": st["M"], "n_lim": args.n_lim,
                          "refine_steps": st["refine_steps"], "precision": args.precision, "batch": B,
                          "cuda_graph": bool(st["graph"]),
                          "prod_direct_max": args.prod_direct_max or "auto",
                          "eval_direct_max": args.eval_direct_max or "auto",
                          "l2": "256 MB flush between steps; working set > L2"},
               "n_solves_per_s": value * n,
               "solves_per_s_per_problem_stream": value / B,
               "normal_eq_rel_residual": res,
               "rel_err_vs_refined": {"value": rel_err_ref, "reference": "same problem, %d FP64 refinement "
                                      "corrections" % nref, "reference_normal_eq_rel_residual": ref_res},
               "e2e": {"value": e2e_v, "unit": "solves/s", "h2d_bytes_per_step": 16 * (2 * m + n),
                       "d2h_bytes_per_step": 16 * n},
               "gpu_launches": int(st["kernel_launches"]) * args.steps,
               "clocks": clocks,
               "peaks": {"hbm_gbs": pk.get("hbm_gbs"), "kind": pk_kind, "fma_fp64_gflops": p64,
                         "fma_fp32_gflops": p32},
               "roofline": roofline,
               "kinds": kr,
               "hbm": {"model_bytes_per_solve": model_bytes_per_solve(st["N"], st["p"]),
                       "achieved_gbs": model_bytes_per_solve(st["N"], st["p"]) * solves_per_item * B / (t_max / 1e3) / 1e9,
                       "pct_of_measured": 100.0 * model_bytes_per_solve(st["N"], st["p"]) * solves_per_item * B
                       / (t_max / 1e3) / 1e9 / pk.get("hbm_gbs", 6788.3)},
               "step_breakdown": breakdown,
               "sweep": sweep,
               "general_problem": general,
               "many_rhs": many,
               "cpu_baseline": cpu}
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
