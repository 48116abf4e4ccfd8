"""One solver for many right-hand sides (tikh_inverse_*): the displacement representation of
(T^H T + lam I)^{-1} built from eight superfast solves on the GPU, against the oracle's representation
(oracle.inverse_generators / inverse_apply, pinned against dense inverses) and dense solves."""
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


def tens(a, cplx):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.complex128 if cplx else torch.float64, device=DEV)


def problem(m, n, lam, cplx, seed):
    return W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, lam, seed=seed, complex_data=cplx, signal="smooth")


@pytest.mark.parametrize("m,n,lam,cplx", [(300, 200, 1e-3, False), (256, 256, 1e-2, True), (1000, 700, 1e-4, True),
                                          (6000, 4096, 1e-3, False)])
def test_generators_and_applies_match_the_oracle_and_dense(m, n, lam, cplx):
    # several FFT tiles and (at n = 4096, N > 4096) the four-step transforms; generators from solves with
    # one refinement correction on both sides
    P = problem(m, n, lam, cplx, seed=m + n)
    col, row = P["col"], P["row"]
    plan = tikh.Plan(m, n, "c128" if cplx else "r64", batch=8, refine_steps=1)
    inv = tikh.Inverse(plan, tens(col, cplx), tens(row, cplx), lam, max_rhs=4)
    g = inv.generators().cpu().numpy()
    u, w = oracle.inverse_generators(col, row, lam)
    ref = np.concatenate([u, w])
    for t in range(8):  # each generator to 1e-9 of its own size
        assert np.abs(g[t] - ref[t]).max() <= 1e-9 * max(np.abs(ref[t]).max(), 1e-300), t
    rng = np.random.default_rng(5)
    R = 3
    y = rng.standard_normal((R, n)) + (1j * rng.standard_normal((R, n)) if cplx else 0.0)
    b = rng.standard_normal((R, m)) + (1j * rng.standard_normal((R, m)) if cplx else 0.0)
    xy = inv.apply(tens(y, cplx), normal=True, refine_steps=0).cpu().numpy()
    xb = inv.apply(tens(b, cplx), normal=False, refine_steps=1).cpu().numpy()
    T = oracle.toeplitz_dense(col, row) if n <= 1000 else None
    for r in range(R):
        if n <= 1000:  # the oracle's plain Hankel sums are O(n^2)
            assert relerr(xy[r], oracle.inverse_apply(u, w, y[r])) <= 1e-10
        if T is not None:
            A = T.conj().T @ T + lam * np.eye(n)
            assert relerr(xy[r], np.linalg.solve(A, y[r])) <= 1e-9
            assert relerr(xb[r], np.linalg.solve(A, T.conj().T @ b[r])) <= 1e-11
        else:
            ys = oracle.apply_th(col, row, b[r])
            xs = oracle.solve_normal_refined(col, row, ys, lam, steps=2)
            assert relerr(xb[r], xs) <= 1e-11


def test_many_right_hand_sides_in_passes_match_one_at_a_time():
    # 7 right-hand sides through passes of 3 (3 + 3 + 1) equal the same right-hand sides one by one, and the
    # plan's own superfast solves
    m, n, lam = 900, 640, 1e-3
    P = problem(m, n, lam, False, seed=11)
    plan = tikh.Plan(m, n, "r64", batch=4, refine_steps=1)
    col, row = tens(P["col"], False), tens(P["row"], False)
    inv = tikh.Inverse(plan, col, row, lam, max_rhs=3)
    b = tens(np.random.default_rng(6).standard_normal((7, m)), False)
    x = inv.apply(b, refine_steps=1).cpu().numpy()
    st = inv.info()
    assert st["kernel_launches"] > 0 and st["workspace_bytes"] > 0
    for r in range(7):
        x1 = inv.apply(b[r].contiguous(), refine_steps=1).cpu().numpy()
        assert relerr(x[r], x1) <= 1e-15
        xs = plan.solve(col, row, b[r].contiguous(), lam).cpu().numpy()
        assert relerr(x[r], xs) <= 1e-10, relerr(x[r], xs)


def test_refinement_corrections_contract():
    # generators from plain superfast solves (no refinement on the plan): the apply alone is as accurate as
    # those solves (the oracle's run of the same steps: 9e-11 from the dense solution), one correction
    # x += X~(y - A x) takes it to rounding level (4e-14 there)
    m, n, lam = 500, 320, 1e-7
    P = W.deconvolution_problem(m, n, 6.0, 30, 1e-6, 1e-6, lam, seed=12, complex_data=True, signal="smooth")
    plan = tikh.Plan(m, n, "c128")
    inv = tikh.Inverse(plan, tens(P["col"], True), tens(P["row"], True), lam, max_rhs=1)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    xd = np.linalg.solve(T.conj().T @ T + lam * np.eye(n), T.conj().T @ P["b"])
    errs = [relerr(inv.apply(tens(P["b"], True), refine_steps=k).cpu().numpy(), xd) for k in (0, 1, 2)]
    assert errs[0] <= 1e-8 and errs[1] <= max(errs[0] / 10, 1e-13) and errs[2] <= 1e-12, errs


def test_c2_shape_apply_matches_the_refined_superfast_solve():
    # the benchmark workload (complex128, m = 98304, n = 65536, lam = 1e-4; N = 163840, four-step):
    # one apply with one correction against the superfast solve with two corrections
    P = W.config_c2()
    m, n, lam = len(P["col"]), len(P["row"]), P["lam"]
    col, row, b = tens(P["col"], True), tens(P["row"], True), tens(P["b"], True)
    plan = tikh.Plan(m, n, "c128", batch=8, refine_steps=1)
    inv = tikh.Inverse(plan, col, row, lam, max_rhs=2)
    x = inv.apply(b, refine_steps=1).cpu().numpy()
    inv.close()
    plan.close()
    ref = tikh.Plan(m, n, "c128", refine_steps=2)
    xr = ref.solve(col, row, b, lam).cpu().numpy()
    ref.close()
    assert relerr(x, xr) <= 1e-9, relerr(x, xr)


def test_inverse_refuses_other_plan_kinds_and_bad_arguments():
    m, n = 40, 30
    P = problem(m, n, 1e-2, False, seed=1)
    col, row = tens(P["col"], False), tens(P["row"], False)
    dual = tikh.Plan(n, m, "r64")  # m < n
    with pytest.raises(tikh.TikhError):
        tikh.Inverse(dual, tens(P["col"][:n], False), tens(np.r_[P["row"], np.zeros(m - n)], False), 1e-2)
    gen = tikh.GeneralPlan(m, n, n)
    with pytest.raises(tikh.TikhError):
        tikh.tikh_inverse_create(gen.h, col.data_ptr(), row.data_ptr(), 1e-2, 2)
    plan = tikh.Plan(m, n, "r64")
    for lam, R in ((0.0, 2), (-1.0, 2), (1e-2, 0), (1e-2, 5000)):
        with pytest.raises(tikh.TikhError):
            tikh.tikh_inverse_create(plan.h, col.data_ptr(), row.data_ptr(), lam, R)
    inv = tikh.Inverse(plan, col, row, 1e-2, max_rhs=2)
    z = torch.zeros((2, m), dtype=torch.float64, device=DEV)
    with pytest.raises(tikh.TikhError):  # strides shorter than the vectors
        tikh.tikh_inverse_apply(inv.h, 2, z.data_ptr(), m - 1, z.data_ptr(), n, 0, 0)
    with pytest.raises(tikh.TikhError):
        tikh.tikh_inverse_apply(inv.h, 1, z.data_ptr(), m, z.data_ptr(), n, 0, 17)
    inv.close()
    for p in (dual, gen, plan):
        p.close()
