"""The Toeplitz-Gramian problem (Sec. 3.4): x = (G + L^H L)^{-1} y on the GPU vs the oracle and dense LAPACK."""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import tikh

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def case(n, pl, cplx, seed, width=8, second_difference=False):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(width) + (1j * rng.standard_normal(width) if cplx else 0.0)
    g = np.array([np.vdot(h[d:], h[:width - d]) if d < width else 0.0 for d in range(n)], dtype=complex)
    if second_difference:  # L = 0.1 x the (n-2) x n second difference [1, -2, 1] (Sec. 7.4's regulariser)
        pl = n - 2
        lcol = np.zeros(pl, complex)
        lcol[0] = 0.1
        lrow = np.zeros(n, complex)
        lrow[:3] = [0.1, -0.2, 0.1]
    else:
        lcol = rng.standard_normal(pl) + (1j * rng.standard_normal(pl) if cplx else 0.0)
        lrow = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
        lrow[0] = lcol[0]
    y = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    if not cplx:
        g, lcol, lrow, y = g.real, lcol.real, lrow.real, y.real
    return g, lcol, lrow, y


def gpu(g, lcol, lrow, y, cplx, **kw):
    dt = torch.complex128 if cplx else torch.float64
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)
    plan = tikh.GramianPlan(len(g), len(lcol), "c128" if cplx else "r64", **kw)
    x = plan.solve(t(g), t(lcol), t(lrow), t(y)).cpu().numpy()
    st = plan.stats()
    plan.close()
    return x, st


@pytest.mark.parametrize("n,pl,cplx,sd", [(7, 3, False, False), (64, 64, True, False), (300, 280, False, False),
                                          (257, 400, True, False), (1000, 0, False, True), (4096, 0, True, True)])
def test_gramian_matches_oracle_and_dense(n, pl, cplx, sd):
    g, lcol, lrow, y = case(n, pl, cplx, seed=n, second_difference=sd)
    x, st = gpu(g, lcol, lrow, y, cplx)
    xo, sto = oracle.solve_gramian(g, lcol, lrow, y, is_complex=int(cplx))
    if not cplx:
        xo = xo.real
    assert (st["N"], st["k"]) == (sto["N"], sto["k"])
    assert relerr(x, xo) <= 1e-9, relerr(x, xo)
    if n <= 1000:
        assert relerr(x, oracle.dense_solve_gramian(g, lcol, lrow, y)) <= 1e-9


def test_gramian_refinement_and_plan_kinds():
    g, lcol, lrow, y = case(2000, 0, False, seed=5, second_difference=True)
    x, st = gpu(g, lcol, lrow, y, False, refine_steps=1)
    assert st["refine_steps"] == 1 and st["rel_residual"] < 1e-12
    assert relerr(x, oracle.dense_solve_gramian(g, lcol, lrow, y)) <= 1e-9
    plan = tikh.GramianPlan(40, 38)
    z = torch.zeros(40, dtype=torch.float64, device=DEV)
    with pytest.raises(tikh.TikhError):  # the l2 entry points refuse a Toeplitz-Gramian plan
        tikh.tikh_solve(plan.h, z.data_ptr(), z.data_ptr(), z.data_ptr(), 1.0, z.data_ptr())
    plan.close()


def test_nufft_gramian_kernel_matches_direct_sums():
    from paper_1302_6945_gb300 import workloads as W
    P = W.nufft_problem(n=1000, K=1300, seed=4)
    t = lambda a, dt: torch.tensor(a, dtype=dt, device=DEV)
    g, y = tikh.nufft_gramian(t(P["f"], torch.float64), t(P["w"], torch.float64), t(P["X"], torch.complex128), 1000)
    go, yo = oracle.nufft_gramian(P["f"], P["w"], P["X"], 1000)
    assert relerr(g.cpu().numpy(), go) <= 1e-12 and relerr(y.cpu().numpy(), yo) <= 1e-12


def test_nufft_reconstruction_n4096():
    # Sec. 7.4's workload: n = K = 4096, cond(G_A + L^H L) ~ 2e7.  The GPU-built Gramian and right-hand side,
    # then the Toeplitz-Gramian solve with two FP64 refinement corrections, against a dense LAPACK solve of the
    # same g and y (inputs identical: at this conditioning their rounding would otherwise dominate)
    from paper_1302_6945_gb300 import workloads as W
    P = W.nufft_problem()
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)
    g, y = tikh.nufft_gramian(t(P["f"], torch.float64), t(P["w"], torch.float64), t(P["X"], torch.complex128), 4096)
    plan = tikh.GramianPlan(4096, 4096, "c128", refine_steps=2)
    lc, lr = t(P["lcol"], torch.complex128), t(P["lrow"], torch.complex128)
    x = plan.solve(g, lc, lr, y).cpu().numpy()
    st = plan.stats()
    plan.close()
    gh, yh = g.cpu().numpy(), y.cpu().numpy()
    xd = oracle.dense_solve_gramian(gh, P["lcol"], P["lrow"], yh)
    assert st["rel_residual"] < 1e-12, st
    assert relerr(x, xd) <= 1e-7, relerr(x, xd)
    assert relerr(x, P["x_true"]) <= 1e-2   # the reconstruction itself (the dense solve's is 2.3e-3)
