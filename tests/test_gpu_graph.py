"""Graph-captured solves (opts.graph = 1) against stream-launched solves of the same plan shape."""
import numpy as np
import pytest
import torch

from paper_1302_6945_gb300 import tikh
from paper_1302_6945_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("m,n,cplx,refine", [(1024, 1024, False, 0), (700, 512, True, 1), (300, 450, False, 0)])
def test_graph_replay_matches_stream_launches(m, n, cplx, refine):
    dt = torch.complex128 if cplx else torch.float64
    P = W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, 1e-3, seed=3, complex_data=cplx)
    t = lambda a: torch.tensor(a, dtype=dt, device=DEV)
    col, row, b = t(P["col"]), t(P["row"]), t(P["b"])
    s = torch.cuda.Stream()  # the legacy default stream cannot be captured
    with torch.cuda.stream(s):
        ref = tikh.Plan(m, n, "c128" if cplx else "r64", refine_steps=refine, stream=s)
        gp = tikh.Plan(m, n, "c128" if cplx else "r64", refine_steps=refine, graph=True, stream=s)
        x = torch.empty(n, dtype=dt, device=DEV)
        for lam in (1e-3, 1e-2, 1e-3):  # capture, then two replays with a new lambda each
            xr = ref.solve(col, row, b, lam).cpu().numpy()
            gp.solve(col, row, b, lam, x=x)
            st = gp.stats()
            assert st["graph"] == 1
            assert relerr(x.cpu().numpy(), xr) <= 1e-14, (lam, relerr(x.cpu().numpy(), xr))
        # new output buffer: the plan captures again
        x2 = gp.solve(col, row, b, 1e-4)
        xr = ref.solve(col, row, b, 1e-4).cpu().numpy()
        assert gp.stats()["graph"] == 1
        assert relerr(x2.cpu().numpy(), xr) <= 1e-14
        # a changed b in the same buffer is seen by the replay
        b.mul_(2.0)
        gp.solve(col, row, b, 1e-4, x=x2)
        xr2 = ref.solve(col, row, b, 1e-4).cpu().numpy()
        assert relerr(x2.cpu().numpy(), xr2) <= 1e-14
        # linear in b only up to the method's forward error (the conditions mix b with data-only
        # entries); a replay that read the old b would be off by 1/2
        assert relerr(x2.cpu().numpy(), 2 * xr) <= 1e-6
        ref.close()
        gp.close()


def test_graph_batched_and_default_stream_fallback():
    m, n, B = 512, 512, 4
    P = W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, 1e-3, seed=7)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV)
    col, row, b = t(P["col"]), t(P["row"]), t(P["b"])
    lams = np.logspace(-4, -1, B)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ref = tikh.Plan(m, n, "r64", batch=B, stream=s)
        gp = tikh.Plan(m, n, "r64", batch=B, graph=True, stream=s)
        xr = ref.solve_strided(col, row, b, lams).cpu().numpy()
        xg = torch.empty((B, n), dtype=torch.float64, device=DEV)
        for _ in range(2):
            gp.solve_strided(col, row, b, lams, x=xg)
            assert gp.stats()["graph"] == 1
            assert relerr(xg.cpu().numpy(), xr) <= 1e-14
        ref.close()
        gp.close()
    # on the legacy default stream capture is impossible: the plan runs stream launches instead
    d = tikh.Plan(m, n, "r64", graph=True, stream=0)
    x = d.solve(col, row, b, 1e-3)
    assert d.stats()["graph"] == 0
    ref = tikh.Plan(m, n, "r64", stream=0)
    assert relerr(x.cpu().numpy(), ref.solve(col, row, b, 1e-3).cpu().numpy()) <= 1e-14
    d.close()
    ref.close()


def test_profiling_by_kind_covers_the_schedule():
    m, n = 1024, 1024
    P = W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, 1e-3, seed=2)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV)
    plan = tikh.Plan(m, n, "r64", graph=True)
    plan.set_profiling(3)
    plan.solve(t(P["col"]), t(P["row"]), t(P["b"]), 1e-3)
    st = plan.stats()
    plan.close()
    assert st["graph"] == 0  # profiled solves run as stream launches
    leaves = st["prof_kind_count"][0]
    assert leaves >= 2 and st["prof_leaf_launches"] == leaves
    assert st["prof_kind_count"][1] == leaves - 1 and st["prof_kind_count"][2] == leaves - 1  # one per inner node
    assert all(v > 0 for v in st["prof_kind_ms"])
    assert abs(st["prof_kind_ms"][0] - st["prof_leaf_ms"]) <= 1e-9 * max(1.0, st["prof_leaf_ms"])
