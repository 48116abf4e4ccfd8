"""Plain CPU FP64 oracle for the superfast Tikhonov solver (arXiv 1302.6945, l2 penalty).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path (``paper_1302_6945_gb300``) never does.
It shares no code with the CUDA library.

Two oracles live here:
  * ``dense_solve`` -- the closed form of Eq. (tiksol): least squares of [T; sqrt(lam) I] x ~ [b; 0]
    by Householder QR (numpy/LAPACK).  Ground truth for small n.
  * the C oracle (``tikh_oracle.c``) -- the paper's algorithm step by step in FP64 (extension,
    transformation, Algorithm 1 with paired interleaving, serial leaves with pivoting, difficult
    points, extraction), with its own textbook DFT.
Beside them, plain numpy for one solver serving many right-hand sides (``inverse_generators``,
``inverse_apply``): the displacement representation of (T^H T + lam I)^{-1}, an extension the paper
does not have, pinned against dense inverses.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tikh_oracle.c")
_SO = os.path.join(_HERE, "_build", "libtikh_oracle.so")

AUTO, DIRECT, FFT = 0, 1, 2


def build(force=False):
    """Compile the C oracle with gcc (plain -O2; no FMA contraction so x86 and Arm agree)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tikh_oracle.h"))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fcx-limited-range", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib_handle = None


class Opts(ctypes.Structure):
    _fields_ = [("nlim", ctypes.c_int), ("m_min", ctypes.c_int), ("eps_diff", ctypes.c_double),
                ("mode", ctypes.c_int), ("fill", ctypes.c_int), ("is_complex", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("M", ctypes.c_int64), ("k", ctypes.c_int64), ("p", ctypes.c_int),
                ("n_difficult", ctypes.c_int64), ("n_dropped", ctypes.c_int64), ("delta", ctypes.c_int * 7),
                ("jstar", ctypes.c_int), ("dual", ctypes.c_int)]

    def as_dict(self, w=5):
        return dict(N=self.N, M=self.M, k=self.k, p=self.p, n_difficult=self.n_difficult,
                    n_dropped=self.n_dropped, delta=list(self.delta)[:w], jstar=self.jstar, dual=self.dual)


def _lib():
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = ctypes.CDLL(build())
    return _lib_handle


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def opts(nlim=32, eps_diff=1e-8, mode=AUTO, m_min=0, fill=0, is_complex=1):
    return Opts(nlim, m_min, eps_diff, mode, fill, is_complex)


def _is_complex(*arrays):
    return int(any(np.iscomplexobj(a) and np.any(np.imag(a) != 0) for a in arrays))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def plan(m, n, nlim=32, m_min=0):
    """Algorithm 2 for the l2 case: returns (N, M, k, p)."""
    N, M, k, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    o = opts(nlim=nlim, m_min=m_min)
    _check(_lib().tikh_oracle_plan(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.byref(o), ctypes.byref(N),
                                   ctypes.byref(M), ctypes.byref(k), ctypes.byref(p)), "plan")
    return N.value, M.value, k.value, p.value


def fft(x, sign=+1):
    """Unnormalised DFT X_k = sum_j x_j exp(sign 2 pi i jk/n)."""
    a = _c128(x).copy()
    _check(_lib().tikh_oracle_fft(ctypes.c_int64(a.size), _ptr(a), ctypes.c_int(sign)), "fft")
    return a


def conditions(col, row, y, lam, nlim=32, m_min=0, fill=0, is_complex=None):
    """(F, G, tau, (N, M, k, p)) for (T^H T + lam I) x = y."""
    if is_complex is None:
        is_complex = _is_complex(col, row)
    col, row, y = _c128(col), _c128(row), _c128(y)
    m, n = col.size, row.size
    pl = plan(m, n, nlim, m_min)
    N = pl[0]
    F = np.zeros((N, 5), np.complex128)
    G = np.zeros((N, 5), np.complex128)
    tau = (ctypes.c_int * 5)()
    o = opts(nlim=nlim, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_conditions(ctypes.c_int64(m), ctypes.c_int64(n), _ptr(col), _ptr(row), _ptr(y),
                                         ctypes.c_double(lam), ctypes.byref(o), _ptr(F), _ptr(G), tau),
           "conditions")
    return F, G, np.array(list(tau)), pl


def leaf(sigma, r, delta, eps=1e-8, cap=None):
    """Serial leaf construction.  Returns dict(B (25, cap), len, order, pivot, deferred, delta, r)."""
    sigma = _c128(sigma)
    r = _c128(r).reshape(-1, 5).copy()
    K = sigma.size
    cap = K + 1 if cap is None else cap
    d = (ctypes.c_int * 5)(*[int(v) for v in delta])
    B = np.zeros((25, cap), np.complex128)
    ln = np.zeros(25, np.int64)
    order = np.zeros(max(K, 1), np.int32)
    piv = np.zeros(max(K, 1), np.int32)
    dq = np.zeros(max(K, 1), np.int32)
    nd = ctypes.c_int()
    _check(_lib().tikh_oracle_leaf(ctypes.c_int(K), _ptr(sigma), _ptr(r), d, ctypes.c_double(eps),
                                   ctypes.c_int64(cap), _ptr(B), _ptr(ln), _ptr(order), _ptr(piv), _ptr(dq),
                                   ctypes.byref(nd)), "leaf")
    return dict(B=B, len=ln, order=order[:K], pivot=piv[:K], deferred=dq[:nd.value], delta=np.array(list(d)), r=r)


def solve_normal(col, row, y, lam, nlim=32, eps_diff=1e-8, mode=AUTO, m_min=0, want_basis=False, fill=0,
                 is_complex=None, want_deferred=False):
    """x = (T^H T + lam I)^{-1} y by the superfast algorithm.  Returns (x, stats[, B, len]); with
    want_deferred, stats["deferred"] lists the ids 2e + f of the conditions deferred as difficult."""
    if is_complex is None:
        is_complex = _is_complex(col, row)
    col, row, y = _c128(col), _c128(row), _c128(y)
    m, n = col.size, row.size
    x = np.zeros(n, np.complex128)
    st = Stats()
    o = opts(nlim=nlim, eps_diff=eps_diff, mode=mode, m_min=m_min, fill=fill, is_complex=is_complex)
    if want_basis:
        cap = plan(m, n, nlim, m_min)[0] + 2
        B = np.zeros((25, cap), np.complex128)
        ln = np.zeros(25, np.int64)
        bp, lp = _ptr(B), _ptr(ln)
    else:
        cap, B, ln, bp, lp = 0, None, None, None, None
    dcap = 2 * plan(m, n, nlim, m_min)[0] if want_deferred else 0
    dq = np.zeros(max(dcap, 1), np.int64)
    rc = _lib().tikh_oracle_solve_normal_ex(ctypes.c_int64(m), ctypes.c_int64(n), _ptr(col), _ptr(row), _ptr(y),
                                            ctypes.c_double(lam), ctypes.byref(o), _ptr(x), ctypes.byref(st), bp,
                                            ctypes.c_int64(cap), lp, _ptr(dq) if want_deferred else None,
                                            ctypes.c_int64(dcap))
    _check(rc, "solve_normal")
    sd = st.as_dict()
    if want_deferred:
        sd["deferred"] = [int(v) for v in dq[:min(sd["n_difficult"], dcap)]]
    if want_basis:
        return x, sd, B, ln
    return x, sd


def solve(col, row, b, lam, nlim=32, eps_diff=1e-8, mode=AUTO, m_min=0, fill=0, is_complex=None):
    """Tikhonov solution argmin ||Tx-b||^2 + lam||x||^2.  Returns (x, stats)."""
    if is_complex is None:
        is_complex = _is_complex(col, row)
    col, row, b = _c128(col), _c128(row), _c128(b)
    m, n = col.size, row.size
    x = np.zeros(n, np.complex128)
    st = Stats()
    o = opts(nlim=nlim, eps_diff=eps_diff, mode=mode, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_solve(ctypes.c_int64(m), ctypes.c_int64(n), _ptr(col), _ptr(row), _ptr(b),
                                    ctypes.c_double(lam), ctypes.byref(o), _ptr(x), ctypes.byref(st)), "solve")
    return x, st.as_dict()


def solve_refined(col, row, b, lam, steps=1, nlim=32, eps_diff=1e-8, mode=AUTO, m_min=0, fill=0, is_complex=None):
    """solve() followed by `steps` refinement corrections.  Returns (x, stats, rel_residual)."""
    if is_complex is None:
        is_complex = _is_complex(col, row)
    col, row, b = _c128(col), _c128(row), _c128(b)
    m, n = col.size, row.size
    x = np.zeros(n, np.complex128)
    st = Stats()
    rr = ctypes.c_double()
    o = opts(nlim=nlim, eps_diff=eps_diff, mode=mode, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_solve_refined(ctypes.c_int64(m), ctypes.c_int64(n), _ptr(col), _ptr(row), _ptr(b),
                                            ctypes.c_double(lam), ctypes.byref(o), ctypes.c_int(steps), _ptr(x),
                                            ctypes.byref(st), ctypes.byref(rr)), "solve_refined")
    return x, st.as_dict(), rr.value


def solve_gramian(g, lcol, lrow, y, nlim=32, eps_diff=1e-8, mode=AUTO, m_min=0, fill=0, is_complex=None):
    """Toeplitz-Gramian problem (Sec. 3.4): x = (G + L^H L)^{-1} y, G Hermitian Toeplitz with first column g,
    L Toeplitz with first column lcol and first row lrow.  Returns (x, stats)."""
    if is_complex is None:
        is_complex = _is_complex(g, lcol, lrow)
    g, lcol, lrow, y = _c128(g), _c128(lcol), _c128(lrow), _c128(y)
    n, pl = g.size, lcol.size
    x = np.zeros(n, np.complex128)
    st = Stats()
    o = opts(nlim=nlim, eps_diff=eps_diff, mode=mode, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_solve_gramian(ctypes.c_int64(n), ctypes.c_int64(pl), _ptr(g), _ptr(lcol), _ptr(lrow),
                                            _ptr(y), ctypes.byref(o), _ptr(x), ctypes.byref(st)), "solve_gramian")
    return x, st.as_dict()


def plan_general(m, n, p, nlim=48, m_min=0):
    """Algorithm 2 with three condition sets per node (Sec. 3.2, 6.2): (N, M, p')."""
    N, M, pp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    o = opts(nlim=nlim, m_min=m_min)
    _check(_lib().tikh_oracle_plan_general(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(p), ctypes.byref(o),
                                           ctypes.byref(N), ctypes.byref(M), ctypes.byref(pp)), "plan_general")
    return N.value, M.value, pp.value


def conditions_general(col, row, lcol, lrow, y, nlim=48, m_min=0, fill=0, is_complex=None):
    """The general problem's interpolation conditions (Eq. (interp)): (cond [N, 3, 7], tau [7])."""
    if is_complex is None:
        is_complex = _is_complex(col, row, lcol, lrow)
    col, row, lcol, lrow, y = _c128(col), _c128(row), _c128(lcol), _c128(lrow), _c128(y)
    m, n, p = col.size, row.size, lcol.size
    N = plan_general(m, n, p, nlim, m_min)[0]
    cond = np.zeros((N, 3, 7), np.complex128)
    tau = (ctypes.c_int * 7)()
    o = opts(nlim=nlim, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_conditions_general(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(p), _ptr(col),
                                                 _ptr(row), _ptr(lcol), _ptr(lrow), _ptr(y), ctypes.byref(o),
                                                 _ptr(cond), tau), "conditions_general")
    return cond, list(tau)


def solve_general(col, row, lcol, lrow, y, nlim=48, eps_diff=1e-12, mode=AUTO, m_min=0, fill=0, is_complex=None):
    """General problem (Sec. 3.2): x = (T^H T + L^H L)^{-1} y with T = [col, row] (m x n) and
    L = [lcol, lrow] (p x n) Toeplitz.  Returns (x, stats).  The difficult-point threshold defaults to
    1e-12: deferring the conditions whose best ratio lies in [1e-12, 1e-8) and processing them against the
    final basis (Sec. 5) cost 1e-7 .. 1e-5 of accuracy on problems of N = 20480 .. 49152 that reach 1e-10
    with them processed in place."""
    if is_complex is None:
        is_complex = _is_complex(col, row, lcol, lrow)
    col, row, lcol, lrow, y = _c128(col), _c128(row), _c128(lcol), _c128(lrow), _c128(y)
    m, n, p = col.size, row.size, lcol.size
    x = np.zeros(n, np.complex128)
    st = Stats()
    o = opts(nlim=nlim, eps_diff=eps_diff, mode=mode, m_min=m_min, fill=fill, is_complex=is_complex)
    _check(_lib().tikh_oracle_solve_general(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(p), _ptr(col),
                                            _ptr(row), _ptr(lcol), _ptr(lrow), _ptr(y), ctypes.byref(o), _ptr(x),
                                            ctypes.byref(st)), "solve_general")
    return x, st.as_dict(w=7)


def dense_solve_general(col, row, lcol, lrow, y):
    """(T^H T + L^H L)^{-1} y by a dense LU solve (numpy)."""
    T = toeplitz_dense(_c128(col), _c128(row))
    L = toeplitz_dense(_c128(lcol), _c128(lrow))
    return np.linalg.solve(T.conj().T @ T + L.conj().T @ L, _c128(y))


def nufft_gramian(f, w, X, n):
    """Sec. 7.4: first column g_d = sum_k w_k exp(+2 pi i f_k d) of the weighted Gramian A^H W A and the
    right-hand side y_s = sum_k w_k X_k exp(+2 pi i f_k s), d, s < n, by the plain direct sums."""
    E = np.exp(2j * np.pi * np.outer(np.arange(n), np.asarray(f, dtype=np.float64)))
    w = np.asarray(w, dtype=np.float64)
    return E @ w, E @ (w * _c128(X))


def hermitian_toeplitz_dense(g):
    """G[i, j] = g_{i-j} with g_{-d} = conj(g_d)."""
    g = _c128(g)
    n = g.size
    return toeplitz_dense(g, np.conj(g))


def dense_solve_gramian(g, lcol, lrow, y):
    """(G + L^H L)^{-1} y by a dense LAPACK solve."""
    G = hermitian_toeplitz_dense(g)
    L = toeplitz_dense(lcol, lrow)
    return np.linalg.solve(G + L.conj().T @ L, _c128(y))


def apply_t(col, row, x):
    col, row, x = _c128(col), _c128(row), _c128(x)
    u = np.zeros(col.size, np.complex128)
    _check(_lib().tikh_oracle_apply_t(ctypes.c_int64(col.size), ctypes.c_int64(row.size), _ptr(col), _ptr(row),
                                      _ptr(x), _ptr(u)), "apply_t")
    return u


def apply_th(col, row, v):
    col, row, v = _c128(col), _c128(row), _c128(v)
    y = np.zeros(row.size, np.complex128)
    _check(_lib().tikh_oracle_apply_th(ctypes.c_int64(col.size), ctypes.c_int64(row.size), _ptr(col), _ptr(row),
                                       _ptr(v), _ptr(y)), "apply_th")
    return y


# ---------------------------------------------------------------------------------------------
# The closed form (Eq. (tiksol)) written out densely.
# ---------------------------------------------------------------------------------------------

def toeplitz_dense(col, row):
    """T[i, j] = a_{i-j}: col[d] = a_d, row[d] = a_{-d} (row[0] ignored)."""
    col, row = _c128(col), _c128(row)
    m, n = col.size, row.size
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    d = i - j
    return np.where(d >= 0, col[np.clip(d, 0, m - 1)], row[np.clip(-d, 0, n - 1)])


def dense_solve(col, row, b, lam):
    """argmin ||Tx - b||^2 + lam ||x||^2 by Householder QR of [T; sqrt(lam) I]."""
    T = toeplitz_dense(col, row)
    m, n = T.shape
    A = np.vstack([T, np.sqrt(lam) * np.eye(n)])
    rhs = np.concatenate([_c128(b), np.zeros(n, np.complex128)])
    Q, Rm = np.linalg.qr(A)
    return np.linalg.solve(Rm, Q.conj().T @ rhs)


def dense_solve_normal(col, row, y, lam):
    """(T^H T + lam I)^{-1} y by a dense LAPACK solve."""
    T = toeplitz_dense(col, row)
    n = T.shape[1]
    return np.linalg.solve(T.conj().T @ T + lam * np.eye(n), _c128(y))


# ---------------------------------------------------------------------------------------------
# Adjoint of x = (T^H T + lam I)^{-1} T^H b, m >= n (conjugate-Wirtinger convention: dL = Re(G^H dx)).
# ---------------------------------------------------------------------------------------------

def solve_normal_refined(col, row, y, lam, steps=1, nlim=32):
    """(T^H T + lam I)^{-1} y by the superfast solve plus `steps` refinement corrections."""
    col, row, y = _c128(col), _c128(row), _c128(y)
    v, _ = solve_normal(col, row, y, lam, nlim=nlim)
    for _ in range(steps):
        res = y - (apply_th(col, row, apply_t(col, row, v)) + lam * v)
        dv, _ = solve_normal(col, row, res, lam, nlim=nlim)
        v = v + dv
    return v


def adjoint(col, row, b, lam, x, G, steps=1, nlim=32):
    """(dL/dcol, dL/drow, dL/db, dL/dlam) for dL/dx = G:  g = A^{-1} G, u = T g, r = b - T x,
    dL/db = u, dL/dlam = -Re(g^H x), dL/da_d = sum_j r_{j+d} conj(g_j) - u_{j+d} conj(x_j)."""
    col, row, b, x, G = _c128(col), _c128(row), _c128(b), _c128(x), _c128(G)
    m, n = col.size, row.size
    g = solve_normal_refined(col, row, G, lam, steps=steps, nlim=nlim)
    u = apply_t(col, row, g)
    r = b - apply_t(col, row, x)
    c = np.correlate(r, g, mode="full") - np.correlate(u, x, mode="full")  # index d + n - 1, d in [-(n-1), m-1]
    dcol = c[n - 1:n - 1 + m]
    drow = np.zeros(n, np.complex128)
    drow[1:] = c[n - 2::-1][:n - 1]
    return dcol, drow, u, float(-np.real(np.vdot(g, x)))


# ---------------------------------------------------------------------------------------------
# One solver for many right-hand sides (an extension: the paper solves one right-hand side per run).
#
# b enters the conditions' fifth component and with it every pivot decision (Sec. 4.3), so the
# interpolation basis of one solve does not serve another right-hand side.  What does carry over is
# the matrix: A = T^H T + lam I (m >= n) has low displacement rank, and so has its inverse.  With Z
# the n x n down-shift ((Z v)_j = v_{j-1}, (Z v)_0 = 0), e_0, f = e_{n-1} and t_d the diagonals of T:
#   A - Z A Z^H = p p^H - q q^H + e_0 s^H + s e_0^H,
#     p_j = conj(t_{-j}),  q_j = conj(t_{m-j}) (q_0 = 0),  s = A e_0 - t_0 p with s_0 halved
# (entries (j, k), j, k >= 1: the sum defining (T^H T)_{jk} minus the same sum shifted by one row of
# T keeps the terms of row 0 and row m of the infinite Toeplitz extension; row and column 0 are
# A's own).  Multiplying Z A Z^H = A - (...) by X = A^{-1} and using Z^H Z = I - f f^H gives
#   X - Z^H X Z = (f - c) a^H + sum_{g in {p, q, e_0, s}} +-(Z^H X g)(X Z^H g')^H ,
# i.e. four rank-one terms (u_t, w_t) built from eight solves X v_i (inverse_rhs below), and since
# Z is nilpotent the Stein equation sums to X = sum_{k<n} (Z^H)^k (X - Z^H X Z) Z^k, that is
#   X y = sum_t H(u_t) H(w_t)^H y,   H(u)_{ik} = u_{i+k} (0 for i + k >= n)  (a Hankel matrix).
# Each term is two correlations, O(n log n) by FFT: after eight solves, every further right-hand
# side of the same T and lam costs a few FFTs instead of a superfast solve.
# ---------------------------------------------------------------------------------------------

def _up(v):  # Z^H v
    return np.concatenate([v[1:], np.zeros(1, np.complex128)])


def _down(v):  # Z v
    return np.concatenate([np.zeros(1, np.complex128), v[:-1]])


def displacement_generators(col, row, lam):
    """p, q, s of A - Z A Z^H = p p^H - q q^H + e_0 s^H + s e_0^H for A = T^H T + lam I (m >= n)."""
    col, row = _c128(col), _c128(row)
    m, n = col.size, row.size
    if m < n:
        raise ValueError("m >= n")
    p = np.conj(np.concatenate([col[:1], row[1:]]))
    q = np.zeros(n, np.complex128)
    q[1:] = np.conj(col[m - np.arange(1, n)])
    e0 = np.zeros(n, np.complex128)
    e0[0] = 1.0
    s = apply_th(col, row, col) + lam * e0 - col[0] * p  # T e_0 is T's first column
    s[0] *= 0.5
    return p, q, s


def inverse_rhs(col, row, lam):
    """The eight right-hand sides v_1..v_8 = f, Z A f, p, q, e_0, Z^H p, Z^H q, Z^H s (m >= n)."""
    col, row = _c128(col), _c128(row)
    n = row.size
    p, q, s = displacement_generators(col, row, lam)
    e0 = np.zeros(n, np.complex128)
    e0[0] = 1.0
    f = np.zeros(n, np.complex128)
    f[-1] = 1.0
    Af = apply_th(col, row, apply_t(col, row, f)) + lam * f
    return [f, _down(Af), p, q, e0, _up(p), _up(q), _up(s)]


def inverse_generators(col, row, lam, solve=None):
    """The four terms (u_t, w_t) with (T^H T + lam I)^{-1} = sum_t H(u_t) H(w_t)^H, as arrays u (4, n), w (4, n).

    solve(y) -> A^{-1} y defaults to the oracle's superfast solve with one refinement correction (Sec. 7.2):
    some of the eight right-hand sides (Z^H s, q: a few entries of T's far diagonals) come out of a plain
    superfast solve 100x less accurate than a data vector does, and their error carries into every apply."""
    if solve is None:
        solve = lambda y: solve_normal_refined(col, row, y, lam, steps=1)
    v = inverse_rhs(col, row, lam)
    xs = [_c128(solve(vi)) for vi in v]
    n = len(v[0])
    f = v[0]
    u = np.stack([f - _up(xs[1]), _up(xs[2]), -_up(xs[3]), _up(xs[4])])
    w = np.stack([xs[0], xs[5], xs[6], xs[7]])
    assert u.shape == (4, n) and w.shape == (4, n)
    return u, w


def hankel_dense(u):
    """H(u)_{ik} = u_{i+k} for i + k < n, else 0."""
    u = _c128(u)
    n = u.size
    i = np.arange(n)[:, None] + np.arange(n)[None, :]
    return np.where(i < n, u[np.clip(i, 0, n - 1)], 0.0)


def inverse_apply(u, w, y):
    """x = sum_t H(u_t) H(w_t)^H y by plain sums: c_k = sum_j conj(w_{j+k}) y_j, x_i = sum_k u_{i+k} c_k."""
    y = _c128(y)
    n = y.size
    x = np.zeros(n, np.complex128)
    for ut, wt in zip(_c128(u), _c128(w)):
        c = np.array([np.vdot(wt[k:], y[:n - k]) for k in range(n)])
        x += np.array([np.dot(ut[i:], c[:n - i]) for i in range(n)])
    return x
