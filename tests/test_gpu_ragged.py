"""Batches of problems of different shapes (tikh_batch_plan_create / tikh_solve_batched) through the C-ABI.

Every item (problem, lambda) is checked against the oracle's refined solve; a budget that forces many
sequential waves and a captured graph must reproduce the one-wave stream result exactly (the per-item
arithmetic does not depend on the wave size or on graph replay).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import tikh
from paper_1302_6945_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problems(shapes, cplx, seed0):
    probs = []
    for i, (m, n) in enumerate(shapes):
        probs.append(W.deconvolution_problem(m, n, 2.0 + i % 5, 12, 1e-6, 1e-6, 1e-3, seed=seed0 + i,
                                             complex_data=cplx, signal="smooth" if cplx else "piecewise"))
    return probs


def _tensors(probs, cplx):
    dt = torch.complex128 if cplx else torch.float64
    t = lambda a: torch.tensor(a, dtype=dt, device=DEV)
    return [t(p["col"]) for p in probs], [t(p["row"]) for p in probs], [t(p["b"]) for p in probs]


# shapes chosen so that several share N (one group) and others do not; one m < n problem
SHAPES = [(300, 200), (310, 190), (290, 211), (700, 512), (650, 560), (120, 90), (90, 120), (1500, 1024)]


@pytest.mark.parametrize("cplx", [False, True])
def test_every_item_matches_the_refined_oracle(cplx):
    probs = _problems(SHAPES, cplx, seed0=40)
    lams = [1e-4, 1e-2, 1.0]
    cols, rows, bs = _tensors(probs, cplx)
    bp = tikh.BatchPlan([p["m"] for p in probs], [p["n"] for p in probs], len(lams), "c128" if cplx else "r64",
                        refine_steps=1)
    xs = bp.solve(cols, rows, bs, lams)
    st = bp.stats()
    bp.close()
    assert st["items"] == len(probs) * len(lams) and 2 <= st["ngroups"] < len(probs)
    for i, P in enumerate(probs):
        for l, lam in enumerate(lams):
            xo, _, _ = oracle.solve_refined(P["col"], P["row"], P["b"], lam, steps=1, is_complex=int(cplx))
            x = xs[i * len(lams) + l].cpu().numpy()
            assert relerr(x, xo if cplx else xo.real) <= 1e-9, (P["m"], P["n"], lam)


def test_waves_and_graph_replay_reproduce_the_one_wave_result():
    probs = _problems(SHAPES, False, seed0=60)
    lams = [1e-3, 1e-1]
    cols, rows, bs = _tensors(probs, False)
    ms, ns = [p["m"] for p in probs], [p["n"] for p in probs]
    one = tikh.BatchPlan(ms, ns, len(lams), "r64")
    x1 = [x.cpu().numpy() for x in one.solve(cols, rows, bs, lams)]
    s1 = one.stats()
    one.close()
    small = tikh.BatchPlan(ms, ns, len(lams), "r64", max_workspace_bytes=s1["workspace_bytes"] // 5)
    s2 = small.stats()
    x2 = [x.cpu().numpy() for x in small.solve(cols, rows, bs, lams)]
    small.close()
    assert s1["max_waves"] == 1 and s2["max_waves"] > 1
    gp = tikh.BatchPlan(ms, ns, len(lams), "r64", graph=True, stream=torch.cuda.Stream())
    with torch.cuda.stream(gp.stream):
        x3 = [x.cpu().numpy() for x in gp.solve(cols, rows, bs, lams)]
        # a second call replays the graph; new right-hand sides in new buffers are seen by the replay
        bs2 = [b * 2.0 for b in bs]
        x4 = [x.cpu().numpy() for x in gp.solve(cols, rows, bs2, lams)]
    torch.cuda.synchronize()
    assert gp.stats()["graph"] == 1
    gp.close()
    for a, b, c, d in zip(x1, x2, x3, x4):
        assert np.array_equal(a, b) and np.array_equal(a, c)
        # x is linear in b, but b enters the conditions' fifth component and with it the pivot scores, so the
        # two solves may pivot differently: they agree to the method's own error
        assert relerr(d, 2.0 * a) <= 1e-8


def test_c3_recipe_sample_as_one_ragged_call():
    # the batching configuration's recipe (first problems of the same seed and draw order) with its
    # 16-value lambda path: small problems vs dense QR, the largest vs the refined oracle
    probs, lams = W.batch_c3(count=16)
    sample = sorted(probs, key=lambda p: p["n"])[:6] + [max(probs, key=lambda p: p["n"])]
    cols, rows, bs = _tensors(sample, False)
    bp = tikh.BatchPlan([p["m"] for p in sample], [p["n"] for p in sample], len(lams), "r64", refine_steps=2,
                        graph=True, stream=torch.cuda.Stream())
    with torch.cuda.stream(bp.stream):
        xs = bp.solve(cols, rows, bs, lams)
    torch.cuda.synchronize()
    bp.close()
    L = len(lams)
    for i, P in enumerate(sample[:3]):
        for l in (0, 7, 15):
            xd = oracle.dense_solve(P["col"], P["row"], P["b"], lams[l]).real
            assert relerr(xs[i * L + l].cpu().numpy(), xd) <= 1e-9, (P["n"], lams[l])
    big = len(sample) - 1
    P = sample[big]
    xo, _, _ = oracle.solve_refined(P["col"], P["row"], P["b"], lams[8], steps=2)
    assert relerr(xs[big * L + 8].cpu().numpy(), xo.real) <= 1e-9


def test_batch_plan_argument_checks():
    with pytest.raises(tikh.TikhError):
        tikh.BatchPlan([10, 0], [5, 5], 2)
    with pytest.raises(tikh.TikhError):
        tikh.BatchPlan([10], [5], 0)
    bp = tikh.BatchPlan([40, 30], [20, 30], 1)
    z = lambda k: torch.zeros(k, dtype=torch.float64, device=DEV)
    with pytest.raises(tikh.TikhError):   # lambda must be > 0
        bp.solve([z(40), z(30)], [z(20), z(30)], [z(40), z(30)], [-1.0])
    bp.close()
