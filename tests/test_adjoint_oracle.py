"""Pins of the adjoint formulas (oracle side, no GPU): PyTorch autograd of the dense closed form and
central finite differences of the oracle solve."""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import workloads as W


def dense_x(col, row, b, lam):
    """x = (T^H T + lam I)^{-1} T^H b from torch tensors (differentiable), T[i,j] = a_{i-j}."""
    m, n = col.shape[0], row.shape[0]
    i = torch.arange(m)[:, None]
    j = torch.arange(n)[None, :]
    d = i - j
    T = torch.where(d >= 0, col[d.clamp(min=0, max=m - 1)], row[(-d).clamp(min=0, max=n - 1)])
    A = T.conj().T @ T + lam * torch.eye(n, dtype=T.dtype)
    return torch.linalg.solve(A, T.conj().T @ b)


@pytest.mark.parametrize("m,n,cplx", [(12, 9, True), (20, 20, False), (33, 17, True), (40, 25, False)])
def test_adjoint_matches_dense_autograd(m, n, cplx):
    P = W.random_problem(m, n, 0.3, seed=m + n, complex_data=cplx)
    dt = torch.complex128 if cplx else torch.float64
    col = torch.tensor(P["col"], dtype=dt, requires_grad=True)
    row = torch.tensor(P["row"], dtype=dt, requires_grad=True)
    b = torch.tensor(P["b"], dtype=dt, requires_grad=True)
    lam = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    x = dense_x(col, row, b, lam)
    rng = np.random.default_rng(1)
    w = torch.tensor(rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0), dtype=dt)
    loss = (w.conj() * x).real.sum() + (x.abs() ** 2).sum()
    loss.backward()
    G = (w + 2 * x).detach().numpy()  # conjugate-Wirtinger gradient of the loss w.r.t. x
    dcol, drow, db, dlam = oracle.adjoint(P["col"], P["row"], P["b"], 0.3, x.detach().numpy(), G, nlim=8)
    if not cplx:
        dcol, drow, db = dcol.real, drow.real, db.real
    gcol = col.grad.numpy().copy()
    grow = row.grad.numpy().copy()
    # the dense matrix reads a_0 from col[0] only; row[0] is ignored (its gradient is 0)
    np.testing.assert_allclose(dcol, gcol, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(drow[1:], grow[1:], rtol=1e-8, atol=1e-10)
    assert abs(grow[0]) == 0.0 and drow[0] == 0
    np.testing.assert_allclose(db, b.grad.numpy(), rtol=1e-8, atol=1e-10)
    assert abs(dlam - lam.grad.item()) <= 1e-8 * max(1.0, abs(dlam))


def test_adjoint_matches_finite_differences():
    P = W.deconvolution_problem(60, 40, 2.0, 8, 1e-3, 1e-3, 0.05, seed=3)
    xt = np.linspace(-1, 1, 40)

    def loss(col, row, b, lam):
        x, _ = oracle.solve(col, row, b, lam, nlim=16, is_complex=0)
        return float(np.sum((x.real - xt) ** 2))

    x, _ = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=16, is_complex=0)
    G = 2 * (x.real - xt)
    dcol, drow, db, dlam = oracle.adjoint(P["col"], P["row"], P["b"], P["lam"], x.real, G, nlim=16)
    h = 1e-6
    fd = (loss(P["col"], P["row"], P["b"], P["lam"] + h) - loss(P["col"], P["row"], P["b"], P["lam"] - h)) / (2 * h)
    assert abs(fd - dlam) <= 1e-5 * max(1.0, abs(dlam))
    for d in (0, 3, 17):
        cp, cm = P["col"].copy(), P["col"].copy()
        cp[d] += h
        cm[d] -= h
        fd = (loss(cp, P["row"], P["b"], P["lam"]) - loss(cm, P["row"], P["b"], P["lam"])) / (2 * h)
        assert abs(fd - dcol[d].real) <= 1e-5 * max(1.0, abs(fd)), d
    for d in (1, 9):
        rp, rm = P["row"].copy(), P["row"].copy()
        rp[d] += h
        rm[d] -= h
        fd = (loss(P["col"], rp, P["b"], P["lam"]) - loss(P["col"], rm, P["b"], P["lam"])) / (2 * h)
        assert abs(fd - drow[d].real) <= 1e-5 * max(1.0, abs(fd)), d
    bp, bm = P["b"].copy(), P["b"].copy()
    bp[5] += h
    bm[5] -= h
    fd = (loss(P["col"], P["row"], bp, P["lam"]) - loss(P["col"], P["row"], bm, P["lam"])) / (2 * h)
    assert abs(fd - db[5].real) <= 1e-5 * max(1.0, abs(fd))
