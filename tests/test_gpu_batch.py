"""Batched solves (tikh_solve_strided) against one-at-a-time solves and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import tikh
from paper_1302_6945_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _single(P, cplx, lam=None, **kw):
    dt = torch.complex128 if cplx else torch.float64
    plan = tikh.Plan(len(P["col"]), len(P["row"]), "c128" if cplx else "r64", **kw)
    t = lambda a: torch.tensor(a, dtype=dt, device=DEV)
    x = plan.solve(t(P["col"]), t(P["row"]), t(P["b"]), P["lam"] if lam is None else lam).cpu().numpy()
    plan.close()
    return x


@pytest.mark.parametrize("m,n,cplx", [(700, 512, False), (512, 512, True), (300, 450, False)])
def test_batch_of_problems_matches_single_solves(m, n, cplx):
    B = 6
    probs = [W.deconvolution_problem(m, n, 3.0 + i, 12 + 2 * i, 1e-6, 1e-6, 10.0 ** (-2 - i % 3), seed=i,
                                     complex_data=cplx, signal="smooth" if cplx else "piecewise") for i in range(B)]
    dt = torch.complex128 if cplx else torch.float64
    col = torch.tensor(np.stack([p["col"] for p in probs]), dtype=dt, device=DEV)
    row = torch.tensor(np.stack([p["row"] for p in probs]), dtype=dt, device=DEV)
    b = torch.tensor(np.stack([p["b"] for p in probs]), dtype=dt, device=DEV)
    lams = [p["lam"] for p in probs]
    # same direct/FFT thresholds on both sides: identical arithmetic per problem
    same = dict(prod_direct_max=36, eval_direct_max=10)
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", batch=B, **same)
    x = plan.solve_strided(col, row, b, lams).cpu().numpy()
    st = plan.stats()
    plan.close()
    # automatic thresholds (a batch plan takes FFT products where a single plan multiplies directly):
    # the same results up to rounding
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", batch=B)
    xa = plan.solve_strided(col, row, b, lams).cpu().numpy()
    plan.close()
    assert st["batch"] == B
    for i, p in enumerate(probs):
        xs = _single(p, cplx, **same)
        assert relerr(x[i], xs) <= 1e-14, (i, relerr(x[i], xs))
        xo, _ = oracle.solve(p["col"], p["row"], p["b"], p["lam"], is_complex=int(cplx))
        xo = xo if cplx else xo.real
        xd = oracle.dense_solve(p["col"], p["row"], p["b"], p["lam"])
        xd = xd if cplx else xd.real
        assert relerr(x[i], xo) <= max(1e-9, 20 * relerr(xo, xd))
        # the two arithmetic variants differ by rounding, amplified as the method's own error is
        xs_auto = _single(p, cplx)
        assert relerr(xa[i], xs_auto) <= max(1e-10, 5 * relerr(xo, xd)), (i, relerr(xa[i], xs_auto))


@pytest.mark.parametrize("m,n,cplx", [(900, 640, False), (400, 600, True)])
def test_several_right_hand_sides_of_one_matrix(m, n, cplx):
    # one T (col and row shared, stride 0) and R right-hand sides: b enters every pivot decision (Sec. 4.3),
    # so each is its own item of one strided batch; each matches its single solve and the dense solution
    R = 5
    P = W.deconvolution_problem(m, n, 4.0, 16, 1e-6, 1e-6, 1e-3, seed=77, complex_data=cplx, signal="smooth")
    rng = np.random.default_rng(78)
    bs = rng.standard_normal((R, m)) + (1j * rng.standard_normal((R, m)) if cplx else 0.0)
    dt = torch.complex128 if cplx else torch.float64
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)
    same = dict(prod_direct_max=36, eval_direct_max=10)
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", batch=R, **same)
    x = plan.solve_strided(t(P["col"]), t(P["row"]), t(bs), [P["lam"]] * R).cpu().numpy()
    plan.close()
    for i in range(R):
        q = dict(P, b=bs[i])
        xs = _single(q, cplx, **same)
        assert relerr(x[i], xs) <= 1e-14, (i, relerr(x[i], xs))
        xd = oracle.dense_solve(P["col"], P["row"], bs[i], P["lam"])
        assert relerr(x[i], xd if cplx else xd.real) <= 1e-9, (i, relerr(x[i], xd))


def test_regularisation_path_shares_generator_and_data():
    # one T and b, 16 lambdas log-spaced 1e-6 .. 1 (the batching workload's path), stride 0 inputs
    P = W.deconvolution_problem(1024, 1024, 4.0, 16, 1e-6, 1e-6, 1.0, seed=5)
    lams = np.logspace(-6, 0, 16)
    plan = tikh.Plan(1024, 1024, "r64", batch=16, refine_steps=1)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=DEV)
    x = plan.solve_strided(t(P["col"]), t(P["row"]), t(P["b"]), lams).cpu().numpy()
    st = plan.stats()
    plan.close()
    assert st["rel_residual"] < 1e-13
    for i, lam in enumerate(lams):
        xd = oracle.dense_solve(P["col"], P["row"], P["b"], lam).real
        assert relerr(x[i], xd) <= 1e-9, (lam, relerr(x[i], xd))


def test_batch_dual_and_refinement():
    B = 3
    probs = [W.deconvolution_problem(400, 600, 3.0, 12, 1e-6, 1e-6, 1e-5, seed=20 + i) for i in range(B)]
    col = torch.tensor(np.stack([p["col"] for p in probs]), device=DEV)
    row = torch.tensor(np.stack([p["row"] for p in probs]), device=DEV)
    b = torch.tensor(np.stack([p["b"] for p in probs]), device=DEV)
    plan = tikh.Plan(400, 600, "r64", batch=4, refine_steps=1)
    x = plan.solve_strided(col, row, b, [p["lam"] for p in probs]).cpu().numpy()
    assert plan.stats()["dual"] == 1
    plan.close()
    for i, p in enumerate(probs):
        xd = oracle.dense_solve(p["col"], p["row"], p["b"], p["lam"]).real
        assert relerr(x[i], xd) <= 1e-9


def test_batch_size_validation():
    plan = tikh.Plan(64, 64, "r64", batch=2)
    z = torch.zeros((3, 64), dtype=torch.float64, device=DEV)
    with pytest.raises(tikh.TikhError):
        plan.solve_strided(z, z, z, [1.0, 1.0, 1.0])
    plan.close()
