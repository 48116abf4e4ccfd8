"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every check here is independent of the oracle's own arithmetic: dense LAPACK solves, closed forms,
numpy's FFT, the defining properties of the interpolation basis (Def. 1, Sec. 4.2-4.3) and the
values the paper prints (Table 1).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1302_6945_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# ----------------------------------------------------------------------------------------------
# DFT
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 12, 60, 97, 128, 240, 1000])
def test_fft_matches_numpy_and_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    # positive sign: evaluation at omega_k = exp(+2 pi i k/n) (Eq. (vandprod))
    np.testing.assert_allclose(oracle.fft(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-12 * n)
    np.testing.assert_allclose(oracle.fft(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * n)
    if n <= 128:
        k = np.arange(n)
        V = np.exp(2j * np.pi * np.outer(k, k) / n)
        np.testing.assert_allclose(oracle.fft(x, +1), V @ x, rtol=0, atol=1e-11 * n)


# ----------------------------------------------------------------------------------------------
# Algorithm 2 (OptExtend), l2 reading: two condition sets, paired interleaving
# ----------------------------------------------------------------------------------------------

def _smooth7(v):
    for f in (2, 3, 5, 7):
        while v % f == 0:
            v //= f
    return v == 1


@pytest.mark.parametrize("m,n,nlim", [(1, 1, 32), (1024, 1024, 32), (98304, 65536, 32), (98304, 65536, 64),
                                      (1572864, 1048576, 32), (327680, 262144, 64), (333, 222, 16),
                                      (5, 700, 8), (257, 1, 32)])
def test_plan_alg2_properties(m, n, nlim):
    N, M, k, p = oracle.plan(m, n, nlim)
    Nt = m + n - 1
    assert N == (M << p) and k == N - Nt and k >= 0          # criteria 1 and 3 (Sec. 6.2)
    assert M % 2 == 0 and _smooth7(M)                        # M even (Sec. 6.2) and 7-smooth (R6)
    # criterion 2 with s = 2 sets: the halving loop stops at the first M with 2M <= N_lim
    Mraw, praw = Nt, 0
    while 2 * Mraw > nlim:
        praw += 1
        Mraw = -(-Mraw // 2)
    assert p == praw and M >= Mraw and M - Mraw < max(8, Mraw // 4)


def test_plan_worked_values():
    # Nt = 2047: 2047 -> 1024 -> 512 -> ... -> 16 after 7 halvings (2*16 <= 32)
    assert oracle.plan(1024, 1024, 32) == (2048, 16, 1, 7)
    # Nt = 163839 -> ceil-halved 14 times to 10 (2*10 <= 32 < 2*20)
    assert oracle.plan(98304, 65536, 32) == (163840, 10, 1, 14)
    # odd M is made even: Nt = 7 with N_lim 100 -> M = 8, k = 1
    assert oracle.plan(4, 4, 100) == (8, 8, 1, 0)


# ----------------------------------------------------------------------------------------------
# Interpolation conditions (Sec. 3.3 + 4.1): the stacked homogeneous system has the Tikhonov
# solution in its null space
# ----------------------------------------------------------------------------------------------

def _stacked_system(F, G, tau, N):
    w = np.exp(2j * np.pi * np.arange(N) / N)
    cols = []
    for i in range(5):
        for t in range(tau[i] + 1):
            cols.append(np.concatenate([F[:, i] * w ** t, G[:, i] * w ** t]))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("m,n,lam,cplx,nlim", [(6, 4, 0.3, True, 8), (9, 9, 1e-2, False, 8), (12, 7, 1e-3, True, 4),
                                               (16, 16, 2.0, True, 16), (21, 13, 1e-4, False, 8)])
def test_conditions_null_space_is_tikhonov_solution(m, n, lam, cplx, nlim):
    P = W.random_problem(m, n, lam, seed=m * 31 + n, complex_data=cplx)
    y = oracle.toeplitz_dense(P["col"], P["row"]).conj().T @ P["b"]
    F, G, tau, (N, M, k, p) = oracle.conditions(P["col"], P["row"], y, lam, nlim=nlim)
    assert list(tau) == [n - 1, m - 1, m + k - 2, n + k - 2, 0]
    A = _stacked_system(F, G, tau, N)
    assert A.shape == (2 * N, 2 * N + 1)
    _, s, vh = np.linalg.svd(A)
    assert s.size == 2 * N and s[-1] > 1e-9 * s[0]   # full row rank: a one-dimensional null space
    v = vh[-1].conj()                                # the right singular vector beyond the 2N values
    assert np.abs(A @ v).max() < 1e-10 * s[0]
    v = v / v[-1]                                    # constant component = 1
    np.testing.assert_allclose(v[:n], oracle.dense_solve(P["col"], P["row"], P["b"], lam), rtol=1e-8, atol=1e-10)
    # sigma_1 = T x (Sec. 3.3): next m coefficients
    T = oracle.toeplitz_dense(P["col"], P["row"])
    np.testing.assert_allclose(v[n:n + m], T @ v[:n], rtol=1e-8, atol=1e-10)


def test_conditions_adjoint_generator_identity():
    # Sec. 7.3: the DFT of the T^H generator follows in O(n) from that of T: lam_H = w^{e(k-1)} conj(t_hat)
    P = W.random_problem(37, 23, 1e-2, seed=3)
    F, G, tau, (N, M, k, p) = oracle.conditions(P["col"], P["row"], np.zeros(23), 1e-2, nlim=8, m_min=12)
    assert k > 1
    e = np.arange(N)
    w = np.exp(2j * np.pi * ((e * (k - 1)) % N) / N)
    np.testing.assert_allclose(F[:, 1], w * np.conj(-G[:, 0]), rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------------------------
# Leaf: serial single-point construction (Eq. (spbasis))
# ----------------------------------------------------------------------------------------------

def _polyval(c, z):
    return np.polyval(c[::-1], z) if len(c) else 0.0


def _Bval(B, ln, z):
    V = np.zeros((5, 5), complex)
    for e in range(25):
        V[e // 5, e % 5] = _polyval(B[e, :ln[e]], z)
    return V


def test_leaf_single_point_is_spbasis():
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    sigma = np.exp(2j * np.pi * 0.3)
    delta = [-3, -5, -5, -2, 0]          # min delta on columns 1, 2: the larger |phi| of them pivots
    out = oracle.leaf([sigma], phi, delta, eps=0.0)
    pi = 1 if abs(phi[1]) > abs(phi[2]) else 2
    assert out["pivot"][0] == pi and list(out["delta"]) == [d + (i == pi) for i, d in enumerate(delta)]
    B = np.zeros((25, 2), complex)
    for i in range(5):
        B[6 * i, 0] = 1.0
    B[6 * pi] = [-sigma, 1.0]                               # (z - sigma) on the pivot
    for i in range(5):
        if i != pi:
            B[5 * pi + i, 0] = -phi[i] / phi[pi]            # mu_i = -phi_i / phi_pi
    np.testing.assert_allclose(out["B"][:, :2], B, rtol=1e-14, atol=1e-15)
    assert np.allclose(phi @ _Bval(out["B"], out["len"], sigma), 0, atol=1e-14)


@pytest.mark.parametrize("K,seed", [(2, 1), (8, 2), (20, 3), (32, 4), (64, 5)])
def test_leaf_basis_properties(K, seed):
    rng = np.random.default_rng(seed)
    sigma = np.exp(2j * np.pi * rng.permutation(4 * K)[:K] / (4 * K))
    phi = rng.standard_normal((K, 5)) + 1j * rng.standard_normal((K, 5))
    phi[::3, 3] = 0.0                                   # structural zeros like F_k, G_k
    delta_in = np.array([-9, -11, -11, -9, 0])
    out = oracle.leaf(sigma, phi.copy(), delta_in, eps=1e-12)
    B, ln, dout = out["B"], out["len"], out["delta"]
    done = [q for q in out["order"] if q >= 0]
    assert len(done) + len(out["deferred"]) == K
    assert (dout - delta_in).sum() == len(done)         # each processed condition raises one degree
    # Def. 1: the basis annihilates every processed condition
    for q in done:
        r = phi[q] @ _Bval(B, ln, sigma[q])
        assert np.abs(r).max() < 1e-9 * np.abs(phi[q]).max() * max(1.0, np.abs(_Bval(B, ln, sigma[q])).max())
    # degree structure: deg B_ij <= delta_out_j - delta_in_i (tau-degree of column j)
    for i in range(5):
        for j in range(5):
            c = B[5 * i + j, :ln[5 * i + j]]
            nz = np.nonzero(np.abs(c) > 0)[0]
            if len(nz):
                assert nz[-1] <= dout[j] - delta_in[i]
    # each elementary factor has determinant (z - sigma): det B(z) = prod over processed (z - sigma_q)
    for z in (0.3 + 0.7j, -1.1 + 0.2j, 2.0):
        ref = np.prod([z - sigma[q] for q in done])
        np.testing.assert_allclose(np.linalg.det(_Bval(B, ln, z)), ref, rtol=1e-9)


def test_leaf_pivot_and_condition_order():
    # two conditions: q0 with a tiny entry in its minimum-degree column, q1 balanced.
    sigma = np.array([1.0, -1.0], complex)
    r = np.array([[1e-3, 1.0, 1.0, 1.0, 1.0], [1.0, 1.0, 0.0, 0.0, 0.0]], complex)
    out = oracle.leaf(sigma, r.copy(), [-2, -1, -1, -1, 0], eps=0.0)
    # column 0 has the minimum degree for both; q1 scores 1/2, q0 scores ~1e-6/4: q1 first (R8)
    assert out["order"][0] == 1 and out["pivot"][0] == 0
    # deferral (R7): with eps above q0's score after the update, q0 is deferred
    out2 = oracle.leaf(sigma, r.copy(), [-2, -1, -1, -1, 0], eps=0.9)
    assert list(out2["deferred"]) == [0, 1]


# ----------------------------------------------------------------------------------------------
# Full solve against the closed form and special cases
# ----------------------------------------------------------------------------------------------

SHAPES = [(1, 1), (2, 1), (1, 2), (5, 3), (3, 5), (17, 17), (64, 40), (40, 64), (100, 100), (131, 77)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("lam", [1e-6, 1e-2, 3.0])
@pytest.mark.parametrize("cplx", [True, False])
def test_solve_matches_dense_qr(m, n, lam, cplx):
    P = W.random_problem(m, n, lam, seed=7 * m + n, complex_data=cplx)
    xd = oracle.dense_solve(P["col"], P["row"], P["b"], lam)
    x, st = oracle.solve(P["col"], P["row"], P["b"], lam, nlim=16)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    cond = np.linalg.cond(T.conj().T @ T + lam * np.eye(n))
    assert relerr(x, xd) <= 1e-13 * cond + 1e-12, (relerr(x, xd), cond)
    assert sorted(st["delta"]) == [0, 1, 1, 1, 1]


@pytest.mark.parametrize("m,n,cplx,eps", [(17, 11, True, 0.2), (40, 27, False, 0.2), (5, 3, True, 0.3),
                                          (11, 17, True, 0.2), (27, 40, False, 0.3)])
def test_difficult_points_processed_at_the_end_match_dense_qr(m, n, cplx, eps):
    # Sec. 5: conditions whose best pivot is too small are deferred and processed serially against the
    # final basis B* (residual Phi_q B*(sigma_q), then single-point steps with no further deferral).
    # A large threshold forces many deferrals; x must still be the Tikhonov solution and the final
    # tau-degrees one 0 and four 1s.  A wrong condition row (F for G), node or transposed B* fails this.
    lam = 1e-2
    P = W.random_problem(m, n, lam, seed=7 * m + n, complex_data=cplx)
    xd = oracle.dense_solve(P["col"], P["row"], P["b"], lam)
    x, st = oracle.solve(P["col"], P["row"], P["b"], lam, nlim=16, eps_diff=eps)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    cond = np.linalg.cond(T.conj().T @ T + lam * np.eye(n))
    assert st["n_difficult"] > 0
    assert relerr(x, xd) <= 1e-13 * cond + 1e-12, (relerr(x, xd), cond, st)
    assert sorted(st["delta"]) == [0, 1, 1, 1, 1]


def test_scalar_closed_form():
    for a, b, lam in [(2.0 + 1j, 0.5 - 3j, 0.7), (-1e-3, 4.0, 1e-6), (0.0, 1.0, 2.0)]:
        x, _ = oracle.solve([a], [a], [b], lam)
        np.testing.assert_allclose(x[0], np.conj(a) * b / (abs(a) ** 2 + lam), rtol=1e-14)


def test_diagonal_closed_form():
    m, n = 12, 9
    col = np.zeros(m, complex)
    col[0] = 1.5 - 0.5j
    row = np.zeros(n, complex)
    row[0] = col[0]
    b = np.arange(m) + 1j
    x, _ = oracle.solve(col, row, b, 0.25, nlim=8)
    np.testing.assert_allclose(x, np.conj(col[0]) * b[:n] / (abs(col[0]) ** 2 + 0.25), rtol=1e-13)


@pytest.mark.parametrize("n,lam", [(16, 1e-3), (60, 0.1), (250, 1e-5)])
def test_circulant_closed_form(n, lam):
    # T circulant with first column c: x = F^{-1}(conj(c_hat) F b / (|c_hat|^2 + lam)) (numpy FFT)
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    row = np.concatenate([[c[0]], c[1:][::-1]])      # a_{-d} = c_{n-d}
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ch = np.fft.fft(c)
    xref = np.fft.ifft(np.conj(ch) * np.fft.fft(b) / (np.abs(ch) ** 2 + lam))
    x, _ = oracle.solve(c, row, b, lam, nlim=16)
    assert relerr(x, xref) < 1e-10


@pytest.mark.parametrize("mode", [oracle.DIRECT, oracle.FFT])
def test_solution_independent_of_leaf_size_extension_and_mode(mode):
    P = W.deconvolution_problem(300, 220, 4.0, 16, 1e-6, 1e-6, 1e-3, seed=11)
    xd = oracle.dense_solve(P["col"], P["row"], P["b"], P["lam"])
    for nlim, m_min in [(8, 0), (16, 0), (32, 0), (64, 0), (16, 12), (32, 20)]:
        x, st = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=nlim, m_min=m_min, mode=mode)
        assert relerr(x, xd) < 1e-9, (nlim, m_min, st)


def test_basis_satisfies_all_conditions():
    # Def. 1 at every node, final degree pattern (Sec. 4.3 end), per-entry degree bound
    P = W.random_problem(45, 31, 1e-2, seed=21)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    y = T.conj().T @ P["b"]
    x, st, B, ln = oracle.solve_normal(P["col"], P["row"], y, 1e-2, nlim=16, want_basis=True)
    F, G, tau, (N, M, k, p) = oracle.conditions(P["col"], P["row"], y, 1e-2, nlim=16)
    assert sorted(st["delta"]) == [0, 1, 1, 1, 1]
    w = np.exp(2j * np.pi * np.arange(N) / N)
    for e in range(N):
        V = _Bval(B, ln, w[e])
        for phi in (F[e], G[e]):
            r = phi @ V
            assert np.abs(r).max() <= 1e-9 * np.abs(phi).max() * np.abs(V).max()
    for i in range(5):
        for j in range(5):
            assert ln[5 * i + j] - 1 <= st["delta"][j] + tau[i]


def test_normal_equation_identity_large():
    P = W.deconvolution_problem(6000, 4096, 4.0, 16, 1e-6, 1e-6, 1e-4, seed=5)
    x, st = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=32)
    r = oracle.apply_th(P["col"], P["row"], P["b"] - oracle.apply_t(P["col"], P["row"], x)) - P["lam"] * x
    assert np.linalg.norm(r) / np.linalg.norm(oracle.apply_th(P["col"], P["row"], P["b"])) < 1e-10
    assert st["n_difficult"] == 0


def test_toeplitz_apply_matches_dense():
    P = W.random_problem(37, 58, 1.0, seed=9)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    x = np.arange(58) * (1 - 0.5j)
    np.testing.assert_allclose(oracle.apply_t(P["col"], P["row"], x), T @ x, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(oracle.apply_th(P["col"], P["row"], P["b"]), T.conj().T @ P["b"], rtol=1e-12,
                               atol=1e-10)


def test_paper_known_x_within_table1_band():
    # Sec. 7.1-7.2: y = (T^H T + |beta|^2 I) x for known x; Table 1 bounds the max error
    band = {}
    with open(os.path.join(GOLDEN, "table1_l2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, v = line.split()
                band[int(n)] = float(v)
    for n in (512, 1024):
        P = W.paper_problem(n, seed=n)
        T = oracle.toeplitz_dense(P["col"], P["row"])
        y = T.conj().T @ (T @ P["x_true"]) + P["lam"] * P["x_true"]
        x, st = oracle.solve_normal(P["col"], P["row"], y, P["lam"], nlim=32)
        assert np.abs(x - P["x_true"]).max() <= 10 * band[n], (n, np.abs(x - P["x_true"]).max())


def test_solution_independent_of_fill():
    # Sec. 6.2: the arbitrary extension entries change only the conditioning, not the solution
    P = W.deconvolution_problem(210, 150, 3.0, 12, 1e-6, 1e-6, 1e-2, seed=4)
    xd = oracle.dense_solve(P["col"], P["row"], P["b"], P["lam"])
    for fill in (0, 1):
        for m_min in (0, 12):
            x, st = oracle.solve(P["col"], P["row"], P["b"], P["lam"], nlim=16, m_min=m_min, fill=fill)
            assert st["k"] > 1 and relerr(x, xd) < 1e-10, (fill, m_min, st["k"], relerr(x, xd))


# ----------------------------------------------------------------------------------------------
# normal-equation form and refinement (Sec. 7.1 right-hand side; Sec. 7.2 refinement)
# ----------------------------------------------------------------------------------------------
def test_solve_normal_matches_dense_normal_equations():
    from scipy.linalg import toeplitz
    rng = np.random.default_rng(11)
    m, n = 300, 200
    col = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    row = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    row[0] = col[0]
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = 0.5
    T = toeplitz(col, row)
    xd = np.linalg.solve(T.conj().T @ T + lam * np.eye(n), y)
    x, _ = oracle.solve_normal(col, row, y, lam)
    assert relerr(x, xd) <= 1e-11


def test_refinement_reaches_dense_accuracy_on_a_smoothing_psf():
    # a strongly smoothing point-spread function at lambda = 1e-6 (the batching recipe's first small
    # problem): the plain method is ~1e-5 from the least-squares solution, two corrections reach the
    # dense solve's own level
    from scipy.linalg import toeplitz
    probs, lams = W.batch_c3(count=24)
    P = [p for p in probs if p["n"] <= 800][0]
    lam = float(lams[0])
    T = toeplitz(P["col"], P["row"])
    A = np.vstack([T, np.sqrt(lam) * np.eye(P["n"])])
    xd = np.linalg.lstsq(A, np.concatenate([P["b"], np.zeros(P["n"])]), rcond=None)[0]
    x0, _ = oracle.solve(P["col"], P["row"], P["b"], lam)
    x2, _, _ = oracle.solve_refined(P["col"], P["row"], P["b"], lam, steps=2)
    assert relerr(x2.real, xd) <= 1e-9
    assert relerr(x2.real, xd) <= 1e-3 * relerr(x0.real, xd)


# ----------------------------------------------------------------------------------------------
# Toeplitz-Gramian problem (Sec. 3.4, Eq. (gramblk), (ex7)): (G + L^H L) x = y
# ----------------------------------------------------------------------------------------------

def _gramian_case(n, pl, cplx, seed, width=8):
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(width) + (1j * rng.standard_normal(width) if cplx else 0.0)
    # G = the autocorrelation Toeplitz of h: Hermitian positive semidefinite, as a Gramian is
    g = np.array([np.vdot(h[d:], h[:width - d]) if d < width else 0.0 for d in range(n)], dtype=complex)
    lcol = rng.standard_normal(pl) + (1j * rng.standard_normal(pl) if cplx else 0.0)
    lrow = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    lrow[0] = lcol[0]
    y = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    return g, lcol, lrow, y


@pytest.mark.parametrize("n,pl,cplx", [(7, 3, False), (20, 20, False), (31, 29, True), (40, 38, False),
                                       (64, 80, True), (50, 10, True), (100, 98, False)])
def test_gramian_matches_dense_solve(n, pl, cplx):
    g, lcol, lrow, y = _gramian_case(n, pl, cplx, seed=n + pl)
    G = oracle.hermitian_toeplitz_dense(g)
    assert np.allclose(G, G.conj().T)
    L = oracle.toeplitz_dense(lcol, lrow)
    A = G + L.conj().T @ L
    xd = np.linalg.solve(A, y)
    x, st = oracle.solve_gramian(g, lcol, lrow, y, nlim=16)
    assert relerr(x, xd) <= 1e-13 * np.linalg.cond(A) + 1e-12, relerr(x, xd)
    assert sorted(st["delta"]) == [0, 1, 1, 1, 1]
    assert st["N"] >= max(n, pl) + n - 1 and st["k"] == st["N"] - (pl + n - 1)


def test_gramian_with_scaled_identity_regulariser_is_a_shifted_toeplitz_solve():
    # L = beta I (pl = n): (G + |beta|^2 I) x = y
    n, beta = 45, 0.7 - 0.2j
    g, _, _, y = _gramian_case(n, n, True, seed=3)
    lcol = np.zeros(n, complex)
    lcol[0] = beta
    lrow = np.zeros(n, complex)
    x, _ = oracle.solve_gramian(g, lcol, lrow, y, nlim=16)
    xd = np.linalg.solve(oracle.hermitian_toeplitz_dense(g) + abs(beta) ** 2 * np.eye(n), y)
    assert relerr(x, xd) <= 1e-12


def test_gramian_with_scaled_identity_gram_is_the_l2_normal_equation():
    # G = lam I: (lam I + L^H L) x = y, the l2 system with T = L (its own pinned solver and dense LAPACK)
    P = W.random_problem(60, 44, 0.3, seed=8)
    y = oracle.apply_th(P["col"], P["row"], P["b"])
    g = np.zeros(44, complex)
    g[0] = 0.3
    x, _ = oracle.solve_gramian(g, P["col"], P["row"], y, nlim=16)
    xn, _ = oracle.solve_normal(P["col"], P["row"], y, 0.3, nlim=16)
    xd = oracle.dense_solve_normal(P["col"], P["row"], y, 0.3)
    assert relerr(x, xd) <= 1e-12 and relerr(xn, xd) <= 1e-12


def test_gramian_solution_independent_of_fill_and_extension():
    g, lcol, lrow, y = _gramian_case(70, 68, False, seed=12)
    xd = oracle.dense_solve_gramian(g, lcol, lrow, y)
    for fill in (0, 1):
        for m_min in (0, 12, 20):
            x, st = oracle.solve_gramian(g, lcol, lrow, y, nlim=16, m_min=m_min, fill=fill)
            assert relerr(x, xd) <= 1e-11, (fill, m_min, st["k"], relerr(x, xd))


def test_nufft_gramian_direct_sums_match_the_matrix_definition():
    # Sec. 7.4: (A^H W A)_{rs} = sum_k w_k exp(2 pi i f_k (r - s)) is Hermitian Toeplitz; g is its first
    # column and y = A^H W X, with A_{ks} = exp(-2 pi i f_k s)
    P = W.nufft_problem(n=48, K=60, seed=2)
    A = np.exp(-2j * np.pi * np.outer(P["f"], np.arange(48)))
    GA = A.conj().T @ np.diag(P["w"]) @ A
    g, y = oracle.nufft_gramian(P["f"], P["w"], P["X"], 48)
    np.testing.assert_allclose(oracle.hermitian_toeplitz_dense(g), GA, rtol=0, atol=1e-13)
    np.testing.assert_allclose(y, A.conj().T @ (P["w"] * P["X"]), rtol=0, atol=1e-12)
    assert abs(P["w"].sum() - 1.0) < 1e-14 and (P["w"] > 0).all()


def test_nufft_reconstruction_small_matches_dense():
    P = W.nufft_problem(n=512, K=512, seed=3)
    g, y = oracle.nufft_gramian(P["f"], P["w"], P["X"], 512)
    xd = oracle.dense_solve_gramian(g, P["lcol"], P["lrow"], y)
    x, _ = oracle.solve_gramian(g, P["lcol"], P["lrow"], y)
    A = oracle.hermitian_toeplitz_dense(g) + oracle.toeplitz_dense(P["lcol"], P["lrow"]).T @ \
        oracle.toeplitz_dense(P["lcol"], P["lrow"])
    assert relerr(x, xd) <= 1e-13 * np.linalg.cond(A) + 1e-12


# ---- the general problem (Sec. 3.2): (T^H T + L^H L) x = y, 7 x 7 basis, conditions F, G, H ----

def _general_case(m, n, p, cplx, seed):
    P = W.general_problem(m, n, p, seed, complex_data=cplx)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    return P, T.conj().T @ P["b"]


@pytest.mark.parametrize("m,n,p,cplx", [(12, 8, 8, False), (30, 20, 20, True), (40, 30, 25, False),
                                        (25, 30, 40, True), (9, 16, 20, False), (100, 64, 64, False),
                                        (301, 200, 150, True), (64, 1, 3, False)])
def test_general_matches_dense_solve(m, n, p, cplx):
    P, y = _general_case(m, n, p, cplx, seed=m + 3 * n + 7 * p)
    T = oracle.toeplitz_dense(P["col"], P["row"])
    L = oracle.toeplitz_dense(P["lcol"], P["lrow"])
    A = T.conj().T @ T + L.conj().T @ L
    xd = np.linalg.solve(A, y)
    x, st = oracle.solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=24)
    assert relerr(x, xd) <= 1e-13 * np.linalg.cond(A) + 1e-12, relerr(x, xd)
    assert st["N"] >= max(m, p) + n - 1 and st["N"] == st["M"] << st["p"]


def test_general_final_degrees_are_six_ones_and_one_zero():
    # Sec. 5: tau sums to 3N - 6, so the final tau-degrees sum to 6 with spread <= 1: six 1s and one 0
    P, y = _general_case(70, 50, 45, True, seed=4)
    cond, tau = oracle.conditions_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=24)
    N = cond.shape[0]
    assert sum(tau) == 3 * N - 6
    x, st = oracle.solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=24)
    assert sorted(st["delta"]) == [0, 1, 1, 1, 1, 1, 1] and st["delta"][st["jstar"]] == 0


@pytest.mark.parametrize("m,n,p", [(7, 5, 6), (10, 8, 12), (14, 9, 9)])
def test_general_conditions_have_the_solution_as_their_only_null_vector(m, n, p):
    # Eq. (ex2)-(interp): the 3N conditions on the 3N + 1 coefficients of p*(z) (component lengths
    # n, m, p, N-n, N-m, N-p, 1) have a one-dimensional null space, spanned by the extended solution;
    # its x part over its constant part is the dense solution
    P, y = _general_case(m, n, p, False, seed=m * n * p)
    cond, tau = oracle.conditions_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=6)
    N = cond.shape[0]
    lens = [t + 1 for t in tau]
    assert lens == [n, m, p, N - n, N - m, N - p, 1]
    w = np.exp(2j * np.pi * np.arange(N) / N)
    cols = []
    for i, L in enumerate(lens):
        V = w[:, None] ** np.arange(L)[None, :]            # N x L monomials at the nodes
        cols.append((cond[:, :, i][:, :, None] * V[:, None, :]).reshape(3 * N, L))
    A = np.concatenate(cols, axis=1)
    assert A.shape == (3 * N, 3 * N + 1)
    s, vh = np.linalg.svd(A)[1:]
    assert s[-1] > 1e-8 * s[0]                             # rank 3N: the null space is one-dimensional
    v = vh[-1].conj()
    xd = oracle.dense_solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y)
    assert relerr(v[:n] / v[-1], xd) <= 1e-10
    assert np.abs(A @ v).max() <= 1e-12 * np.abs(A).max()


def test_general_with_scaled_identity_regulariser_is_the_l2_solve():
    # L = beta I (p = n): T^H T + |beta|^2 I, the l2 system of Sec. 3.3 (its own pinned solver)
    P, y = _general_case(60, 44, 44, True, seed=8)
    beta = 0.6 + 0.3j
    lcol = np.zeros(44, complex)
    lcol[0] = beta
    x, _ = oracle.solve_general(P["col"], P["row"], lcol, np.zeros(44, complex), y, nlim=24)
    xn, _ = oracle.solve_normal(P["col"], P["row"], y, abs(beta) ** 2, nlim=16)
    xd = oracle.dense_solve_normal(P["col"], P["row"], y, abs(beta) ** 2)
    assert relerr(x, xd) <= 1e-12 and relerr(xn, xd) <= 1e-12


def test_general_second_difference_regulariser():
    # the scaled second-order difference L of Sec. 7.4 (p = n, stencil [-1, 2, -1])
    P, y = _general_case(90, 64, 64, False, seed=11)
    lcol = np.zeros(64)
    lcol[:2] = [2.0, -1.0]
    x, _ = oracle.solve_general(P["col"], P["row"], lcol, lcol.copy(), y, nlim=24)
    xd = oracle.dense_solve_general(P["col"], P["row"], lcol, lcol, y)
    assert relerr(x, xd) <= 1e-11


def test_general_solution_independent_of_fill_extension_and_mode():
    P, y = _general_case(80, 56, 50, False, seed=13)
    xd = oracle.dense_solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y)
    for fill in (0, 1):
        for m_min in (0, 14, 24):
            for mode in (oracle.AUTO, oracle.DIRECT, oracle.FFT):
                x, st = oracle.solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=24, m_min=m_min,
                                             fill=fill, mode=mode)
                assert relerr(x, xd) <= 1e-11, (fill, m_min, mode, st["N"], relerr(x, xd))


@pytest.mark.parametrize("m,n,p,eps", [(30, 20, 25, 0.2), (17, 11, 11, 0.3), (40, 27, 30, 0.25)])
def test_general_difficult_points_processed_at_the_end_match_dense(m, n, p, eps):
    # Sec. 5 with a large threshold: many conditions deferred, the result still the exact solution
    P, y = _general_case(m, n, p, True, seed=m + n + p)
    xd = oracle.dense_solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y)
    x, st = oracle.solve_general(P["col"], P["row"], P["lcol"], P["lrow"], y, nlim=24, eps_diff=eps)
    assert st["n_difficult"] > 0
    assert relerr(x, xd) <= 1e-10, (st, relerr(x, xd))


@pytest.mark.parametrize("K,delta_in,seed", [(8, [-10, -10, 0, 0, 0], 1), (12, [-30, -9, -9, -30, 0], 2),
                                             (6, [-4, -20, -4, -4, -4], 3)])
def test_rows_of_unpivoted_columns_stay_identity_rows(K, delta_in, seed):
    # Eq. (spbasis): a single-point factor changes only its pivot column and its rows other than the pivot's
    # are identity rows, so in a basis built from several factors every row of a column that was never a
    # pivot is exactly e_i (the GPU's evaluations and products rely on this to skip those rows)
    rng = np.random.default_rng(seed)
    sigma = np.exp(2j * np.pi * rng.permutation(4 * K)[:K] / (4 * K))
    phi = rng.standard_normal((K, 5)) + 1j * rng.standard_normal((K, 5))
    out = oracle.leaf(sigma, phi.copy(), delta_in, eps=1e-12)
    pivoted = set(int(p) for p in out["pivot"][:K])
    unpivoted = [i for i in range(5) if i not in pivoted]
    assert unpivoted and all(out["delta"][i] == delta_in[i] for i in unpivoted)
    B, ln = out["B"], out["len"]
    for i in unpivoted:
        for j in range(5):
            e = B[5 * i + j, :ln[5 * i + j]]
            if j == i:
                assert ln[5 * i + j] >= 1 and e[0] == 1.0 and not np.any(e[1:])
            else:
                assert not np.any(e)


# ---- one solver for many right-hand sides: the displacement representation of (T^H T + lam I)^{-1} ----

def _rand_toeplitz(m, n, cplx, seed):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(m) + (1j * rng.standard_normal(m) if cplx else 0.0)
    r = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
    r[0] = c[0]
    return c, r


@pytest.mark.parametrize("m,n,cplx", [(7, 5, False), (30, 20, True), (16, 16, False), (40, 9, True)])
def test_displacement_of_the_normal_matrix(m, n, cplx):
    # A - Z A Z^H written out densely against p p^H - q q^H + e_0 s^H + s e_0^H
    col, row = _rand_toeplitz(m, n, cplx, m + n)
    lam = 0.37
    T = oracle.toeplitz_dense(col, row)
    A = T.conj().T @ T + lam * np.eye(n)
    Z = np.eye(n, k=-1)
    p, q, s = oracle.displacement_generators(col, row, lam)
    e0 = np.eye(n)[0]
    D = np.outer(p, p.conj()) - np.outer(q, q.conj()) + np.outer(e0, s.conj()) + np.outer(s, e0)
    assert np.abs((A - Z @ A @ Z.T) - D).max() <= 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("m,n,cplx", [(7, 5, False), (30, 20, True), (16, 16, True), (40, 9, False)])
def test_inverse_is_the_sum_of_four_hankel_products(m, n, cplx):
    # with exact solves: the Stein-equation terms against the dense inverse, matrix by matrix
    col, row = _rand_toeplitz(m, n, cplx, 3 * m + n)
    lam = 0.5
    T = oracle.toeplitz_dense(col, row)
    A = T.conj().T @ T + lam * np.eye(n)
    X = np.linalg.inv(A)
    u, w = oracle.inverse_generators(col, row, lam, solve=lambda y: np.linalg.solve(A, y))
    Z = np.eye(n, k=-1)
    D = sum(np.outer(u[t], w[t].conj()) for t in range(4))
    assert np.abs(D - (X - Z.T @ X @ Z)).max() <= 1e-12 * np.abs(X).max()
    H = lambda v: oracle.hankel_dense(v)
    Xr = sum(H(u[t]) @ H(w[t]).conj().T for t in range(4))
    assert np.abs(Xr - X).max() <= 1e-12 * np.abs(X).max()
    y = np.random.default_rng(1).standard_normal(n) + 0j
    assert np.linalg.norm(oracle.inverse_apply(u, w, y) - X @ y) <= 1e-12 * np.linalg.norm(X @ y)


def test_inverse_generators_of_a_scaled_identity():
    # T = 0: A = lam I, the only term is (f, f / lam), and sum_k (Z^H)^k f f^H Z^k / lam = I / lam
    n, lam = 9, 0.25
    u, w = oracle.inverse_generators(np.zeros(12), np.zeros(n), lam, solve=lambda y: y / lam)
    f = np.eye(n)[-1]
    assert np.allclose(u[0], f, atol=0) and np.allclose(w[0], f / lam, atol=0)
    assert not np.any(u[1:] * 0 != 0) and np.abs(u[1:]).max() * np.abs(w[1:]).max() == 0.0
    y = np.arange(1.0, n + 1)
    assert np.allclose(oracle.inverse_apply(u, w, y), y / lam, rtol=1e-15, atol=0)


@pytest.mark.parametrize("m,n,cplx,lam", [(300, 200, False, 1e-3), (256, 256, True, 1e-2)])
def test_inverse_from_superfast_solves_matches_dense(m, n, cplx, lam):
    # the generators from the oracle's (refined) superfast solves: every right-hand side through the
    # Hankel sums lands within 1e-11 of the dense solution (condition numbers 1e3 and 20 here); from
    # unrefined solves (errors up to 4e-8 on the hardest generator) one correction x += X~(y - A x)
    # with the same sums does the same
    P = W.deconvolution_problem(m, n, 3.0, 12, 1e-6, 1e-6, lam, seed=n, complex_data=cplx, signal="smooth")
    col, row = P["col"], P["row"]
    u, w = oracle.inverse_generators(col, row, lam)
    u0, w0 = oracle.inverse_generators(col, row, lam, solve=lambda y: oracle.solve_normal(col, row, y, lam)[0])
    A = lambda v: oracle.apply_th(col, row, oracle.apply_t(col, row, v)) + lam * v
    rng = np.random.default_rng(2)
    for _ in range(3):
        y = rng.standard_normal(n) + (1j * rng.standard_normal(n) if cplx else 0.0)
        xd = oracle.dense_solve_normal(col, row, y, lam)
        err = lambda v: np.linalg.norm(v - xd) / np.linalg.norm(xd)
        assert err(oracle.inverse_apply(u, w, y)) <= 1e-11
        x0 = oracle.inverse_apply(u0, w0, y)
        assert err(x0 + oracle.inverse_apply(u0, w0, y - A(x0))) <= 1e-11
