"""The failure statuses of include/tikh.h, each made to fire from the host side without faulting or
hanging the GPU, and the plan still usable afterwards.

- TIKH_EDIFFICULT: a deferred-condition list of one entry and a threshold that defers many (Sec. 5).
- TIKH_ENUMERIC: a NaN or Inf in col, row or b; the prologue's check marks the problem and its leaves
  process nothing, so no kernel iterates on non-finite values.
- TIKH_ETIMEOUT: the leaf's one in-kernel wait (its rebuild warps polling for the next pivot step) given
  a limit of one poll; it gives up, records the status and the kernel returns normally.
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _tensors(P, cplx=False):
    dt = torch.complex128 if cplx else torch.float64
    return [torch.tensor(P[k], dtype=dt, device=DEV) for k in ("col", "row", "b")]


def _good_solve_after(plan, P):
    col, row, b = _tensors(P)
    x = plan.solve(col, row, b, P["lam"]).cpu().numpy()
    xo, _ = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=plan.opts.n_lim, is_complex=0)
    assert relerr(x, xo.real) <= 1e-9


def test_too_many_difficult_points_returns_edifficult():
    P = W.random_problem(200, 150, 1e-2, seed=9, complex_data=False)
    col, row, b = _tensors(P)
    plan = tikh.Plan(200, 150, "r64", n_lim=16, eps_diff=0.3, max_difficult=1)
    with pytest.raises(tikh.TikhError) as e:
        plan.solve(col, row, b, P["lam"])
    assert e.value.status == tikh.TIKH_EDIFFICULT
    cnt, _ = plan.difficult()
    assert cnt > 1
    plan.close()


@pytest.mark.parametrize("where,value", [("col", float("nan")), ("row", float("inf")), ("b", float("-inf")),
                                         ("b", float("nan"))])
def test_non_finite_input_returns_enumeric(where, value):
    P = W.random_problem(120, 90, 1e-2, seed=4, complex_data=False)
    bad = dict(P)
    bad[where] = np.array(P[where], copy=True)
    bad[where][3] = value
    col, row, b = _tensors(bad)
    plan = tikh.Plan(120, 90, "r64", n_lim=16)
    with pytest.raises(tikh.TikhError) as e:
        plan.solve(col, row, b, P["lam"])
    assert e.value.status == tikh.TIKH_ENUMERIC
    _good_solve_after(plan, P)   # the status is cleared and the next solve is correct
    plan.close()


def test_non_finite_entry_of_one_problem_in_a_batch_is_reported():
    P = W.random_problem(64, 48, 1e-2, seed=5, complex_data=True)
    col, row, b = _tensors(P, cplx=True)
    B = 3
    cb = col.repeat(B, 1).contiguous()
    cb[1, 7] = complex(float("nan"), 0.0)
    plan = tikh.Plan(64, 48, "c128", n_lim=16, batch=B)
    with pytest.raises(tikh.TikhError) as e:
        plan.solve_strided(cb, row, b, [P["lam"]] * B)
    assert e.value.status == tikh.TIKH_ENUMERIC
    plan.close()


def test_wait_that_gives_up_returns_etimeout():
    P = W.random_problem(120, 90, 1e-2, seed=6, complex_data=False)
    col, row, b = _tensors(P)
    plan = tikh.Plan(120, 90, "r64", n_lim=16, wait_polls=1)
    with pytest.raises(tikh.TikhError) as e:
        plan.solve(col, row, b, P["lam"])
    assert e.value.status == tikh.TIKH_ETIMEOUT
    plan.close()
    plan = tikh.Plan(120, 90, "r64", n_lim=16)   # the context is intact: a normal plan solves correctly
    _good_solve_after(plan, P)
    plan.close()
