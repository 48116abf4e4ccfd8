"""The library's hand-written adjoint (tikh_solve_grad) and the autograd Function on the GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import tikh
from paper_1302_6945_gb300 import workloads as W

from test_adjoint_oracle import dense_x

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("m,n,cplx", [(120, 90, True), (300, 200, False), (1024, 1024, False), (700, 512, True)])
def test_library_adjoint_matches_oracle_adjoint(m, n, cplx):
    P = W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, 1e-3, seed=m, complex_data=cplx,
                                signal="smooth" if cplx else "piecewise")
    dt = torch.complex128 if cplx else torch.float64
    t = lambda a: torch.tensor(a, dtype=dt, device=DEV)
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", refine_steps=1)
    col, row, b = t(P["col"]), t(P["row"]), t(P["b"])
    x = plan.solve(col, row, b, P["lam"])
    rng = np.random.default_rng(m)
    G = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0)
    dcol, drow, db, dlam = plan.grad(col, row, b, P["lam"], x, t(G))
    plan.close()
    ocol, orow, ob, olam = oracle.adjoint(P["col"], P["row"], P["b"], P["lam"], x.cpu().numpy(), G)
    if not cplx:
        ocol, orow, ob = ocol.real, orow.real, ob.real
    assert relerr(dcol.cpu().numpy(), ocol) <= 1e-9
    assert relerr(drow.cpu().numpy(), orow) <= 1e-9
    assert relerr(db.cpu().numpy(), ob) <= 1e-9
    assert abs(dlam - olam) <= 1e-9 * max(1.0, abs(olam))


def test_autograd_function_matches_dense_gradient_n512():
    # the differentiation workload's dense check: loss ||x - x_true||^2 at n = 512
    P = W.deconvolution_problem(640, 512, 4.0, 16, 1e-6, 1e-6, 1e-3, seed=7)
    plan = tikh.Plan(640, 512, "r64", refine_steps=1)
    col = torch.tensor(P["col"], device=DEV, requires_grad=True)
    row = torch.tensor(P["row"], device=DEV, requires_grad=True)
    b = torch.tensor(P["b"], device=DEV, requires_grad=True)
    lam = torch.tensor(P["lam"], device=DEV, requires_grad=True)
    xt = torch.tensor(P["x_true"], device=DEV)
    x = tikh.tikh_solve_autograd(col, row, b, lam, plan)
    ((x - xt) ** 2).sum().backward()
    plan.close()
    c2 = torch.tensor(P["col"], requires_grad=True)
    r2 = torch.tensor(P["row"], requires_grad=True)
    b2 = torch.tensor(P["b"], requires_grad=True)
    l2 = torch.tensor(P["lam"], requires_grad=True)
    x2 = dense_x(c2, r2, b2, l2)
    ((x2 - torch.tensor(P["x_true"])) ** 2).sum().backward()
    assert relerr(x.detach().cpu().numpy(), x2.detach().numpy()) <= 1e-9
    assert relerr(col.grad.cpu().numpy(), c2.grad.numpy()) <= 1e-8
    assert relerr(row.grad.cpu().numpy()[1:], r2.grad.numpy()[1:]) <= 1e-8
    assert relerr(b.grad.cpu().numpy(), b2.grad.numpy()) <= 1e-8
    assert abs(lam.grad.item() - l2.grad.item()) <= 1e-8 * abs(l2.grad.item())


def test_lambda_gradient_matches_central_difference_on_gpu():
    P = W.deconvolution_problem(2000, 1500, 5.0, 20, 1e-6, 1e-6, 1e-2, seed=11)
    plan = tikh.Plan(2000, 1500, "r64", refine_steps=1)
    t = lambda a: torch.tensor(a, device=DEV)
    col, row, b, xt = t(P["col"]), t(P["row"]), t(P["b"]), t(P["x_true"])
    loss = lambda lam: float(((plan.solve(col, row, b, lam) - xt) ** 2).sum())
    x = plan.solve(col, row, b, P["lam"])
    _, _, _, dlam = plan.grad(col, row, b, P["lam"], x, 2 * (x - xt))
    h = 1e-6 * P["lam"]
    fd = (loss(P["lam"] + h) - loss(P["lam"] - h)) / (2 * h)
    plan.close()
    assert abs(fd - dlam) <= 1e-5 * abs(dlam)


@pytest.mark.parametrize("cplx", [False, True])
def test_strided_batch_adjoint_matches_oracle(cplx):
    B, m, n = 4, 300, 200
    probs = [W.deconvolution_problem(m, n, 3.0 + i, 12, 1e-6, 1e-6, 1e-3 * (i + 1), seed=90 + i, complex_data=cplx,
                                     signal="smooth" if cplx else "piecewise") for i in range(B)]
    dt = torch.complex128 if cplx else torch.float64
    t = lambda a: torch.tensor(np.stack(a), dtype=dt, device=DEV)
    col, row, b = t([p["col"] for p in probs]), t([p["row"] for p in probs]), t([p["b"] for p in probs])
    lams = [p["lam"] for p in probs]
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", refine_steps=1, batch=B)
    x = plan.solve_strided(col, row, b, lams)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((B, n)) + (1j * rng.standard_normal((B, n)) if cplx else 0)
    dcol, drow, db, dlam = plan.grad_strided(col, row, b, lams, x, torch.tensor(G, dtype=dt, device=DEV))
    plan.close()
    for i, P in enumerate(probs):
        ocol, orow, ob, olam = oracle.adjoint(P["col"], P["row"], P["b"], P["lam"], x[i].cpu().numpy(), G[i])
        if not cplx:
            ocol, orow, ob = ocol.real, orow.real, ob.real
        assert relerr(dcol[i].cpu().numpy(), ocol) <= 1e-9
        assert relerr(drow[i].cpu().numpy(), orow) <= 1e-9
        assert relerr(db[i].cpu().numpy(), ob) <= 1e-9
        assert abs(dlam[i] - olam) <= 1e-9 * max(1.0, abs(olam))
