"""The benchmark's own accuracy checks (FFT Toeplitz products in torch on the CPU) against dense algebra."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1302_6945_gb300 import workloads as W  # noqa: E402


def test_toeplitz_products_match_the_dense_matrix():
    rng = np.random.default_rng(4)
    for m, n in ((37, 58), (64, 9), (1, 5), (40, 40)):
        col = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        row = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        row[0] = col[0]
        T = oracle.toeplitz_dense(col, row)
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        t = lambda a: torch.tensor(a, dtype=torch.complex128)
        np.testing.assert_allclose(bench.toeplitz_mv_t(torch, t(col), t(row), t(x)).numpy(), T @ x, atol=1e-12)
        np.testing.assert_allclose(bench.toeplitz_mv_t(torch, t(col), t(row), t(v), True).numpy(), T.conj().T @ v,
                                   atol=1e-12)


def test_general_residual_of_the_dense_solution_is_rounding_and_of_a_perturbed_one_is_not():
    P = W.general_problem(90, 64, 70, seed=3)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    xd = oracle.dense_solve_general(P["col"], P["row"], P["lcol"], P["lrow"], T.T @ P["b"]).real
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    args = [t(P[k]) for k in ("col", "row", "lcol", "lrow", "b")]
    assert bench.general_residual_t(torch, *args, t(xd)) < 1e-12
    assert bench.general_residual_t(torch, *args, t(xd * (1 + 1e-6))) > 1e-8


def test_normal_residual_of_the_dense_solution_is_rounding():
    P = W.random_problem(80, 50, 0.3, seed=6)
    xd = oracle.dense_solve(P["col"], P["row"], P["b"], 0.3)
    t = lambda a: torch.tensor(a, dtype=torch.complex128)
    assert bench.normal_residual_t(torch, t(P["col"]), t(P["row"]), t(P["b"]), t(xd), 0.3) < 1e-12
