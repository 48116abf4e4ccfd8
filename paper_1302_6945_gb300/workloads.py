"""Seeded synthetic inputs shaped like the benchmark workloads.

This module holds no arithmetic of the solver: it draws generators, signals and noise, and forms
the data b = T x_true + noise with a library convolution.  Both the CUDA path and the CPU oracle
are fed from here, so they see identical bytes.

Readings of the workload descriptions (all inputs synthetic; no dataset exists for this paper):
  * "discretised Gaussian PSF (sigma s, support +-w)": a_d = exp(-d^2 / 2 s^2) / sum, |d| <= w,
    zero outside; w = ceil(4 s) when the support is not given.  Noise of the stated standard
    deviation is added i.i.d. to every one of the m+n-1 diagonals.
  * complex workloads multiply each PSF tap by an independent unit-modulus phase exp(i theta_d),
    theta_d ~ U[0, 2 pi), and draw complex noise with the stated deviation per real/imag part.
  * "piecewise constant with 8 random jumps": 8 distinct jump positions in [1, n-1], levels N(0,1).
  * "complex Gaussian smoothed by a width-32 box": same-size moving average of width 32.
  * the paper-shaped workload (Sec. 7.1-7.2): complex standard-normal square T, known x,
    y = (T^H T + lam I) x with lam = |beta|^2 = sqrt(N), N read as m + n.
"""
import math

import numpy as np


def gaussian_psf_generator(m, n, sigma, support, noise, rng, complex_phase=False):
    """Return (col, row) with col[d] = a_d (d >= 0), row[d] = a_{-d}; row[0] = col[0]."""
    d = np.arange(-(n - 1), m)
    a = np.exp(-(d.astype(np.float64) ** 2) / (2.0 * sigma * sigma)) * (np.abs(d) <= support)
    a = a / a.sum()
    if complex_phase:
        a = a * np.exp(2j * np.pi * rng.random(a.size))
        a = a + noise * (rng.standard_normal(a.size) + 1j * rng.standard_normal(a.size))
    else:
        a = a + noise * rng.standard_normal(a.size)
    col = a[n - 1:].copy()
    row = a[:n][::-1].copy()
    row[0] = col[0]
    return col, row


def toeplitz_matvec(col, row, x):
    """T x via a library convolution of the diagonal sequence with x (input generation only)."""
    m, n = len(col), len(row)
    a = np.concatenate([np.asarray(row)[1:][::-1], np.asarray(col)])  # a_{-(n-1)} .. a_{m-1}
    L = 1 << int(math.ceil(math.log2(a.size + n)))
    full = np.fft.ifft(np.fft.fft(a, L) * np.fft.fft(np.asarray(x), L))
    out = full[n - 1:n - 1 + m]
    if np.isrealobj(col) and np.isrealobj(row) and np.isrealobj(x):
        out = out.real
    return out


def piecewise_constant(n, jumps, rng):
    pos = np.sort(rng.choice(np.arange(1, n), size=min(jumps, n - 1), replace=False))
    x = np.zeros(n)
    edges = np.concatenate([[0], pos, [n]])
    for i in range(len(edges) - 1):
        x[edges[i]:edges[i + 1]] = rng.standard_normal()
    return x


def box_smooth(x, width):
    k = np.ones(width) / width
    return np.convolve(x, k, mode="same")


def deconvolution_problem(m, n, sigma, support, gen_noise, data_noise, lam, seed, complex_data=False,
                          signal="piecewise"):
    """One deconvolution-shaped problem: dict(col, row, b, lam, x_true)."""
    rng = np.random.default_rng(seed)
    col, row = gaussian_psf_generator(m, n, sigma, support, gen_noise, rng, complex_phase=complex_data)
    if signal == "piecewise":
        x = piecewise_constant(n, 8, rng)
    else:
        x = rng.standard_normal(n) + (1j * rng.standard_normal(n) if complex_data else 0.0)
        x = box_smooth(x, 32)
    b = toeplitz_matvec(col, row, x)
    if complex_data:
        b = b + data_noise * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
    else:
        b = b + data_noise * rng.standard_normal(m)
    return dict(col=col, row=row, b=b, lam=lam, x_true=x, m=m, n=n)


def config_c1(seed=0):
    """m = n = 1024, real, PSF sigma 4 support +-16, 1e-6 generator noise, lam 1e-3."""
    return deconvolution_problem(1024, 1024, 4.0, 16, 1e-6, 1e-6, 1e-3, seed)


def config_c2(seed=1, m=98304, n=65536):
    """complex128, m = 98304, n = 65536, PSF sigma 8 with random phases, lam 1e-4."""
    return deconvolution_problem(m, n, 8.0, 32, 1e-6, 1e-4, 1e-4, seed, complex_data=True, signal="smooth")


def config_c4(seed=3, m=1572864, n=1048576):
    """real, m = 1572864, n = 1048576, PSF sigma 12, 1e-7 generator noise, lam 1e-5."""
    return deconvolution_problem(m, n, 12.0, 48, 1e-7, 1e-7, 1e-5, seed)


def config_c5(seed=4, m=327680, n=262144):
    """real, m = 327680, n = 262144, PSF sigma 8, lam 1e-3 (the differentiation configuration; the loss
    is ||x - x_true||^2)."""
    return deconvolution_problem(m, n, 8.0, 32, 1e-6, 1e-6, 1e-3, seed)


def sweep_problem(n, seed=5):
    """metric sweep point: n = 2^e, m = 1.5 n, PSF sigma 8, real."""
    return deconvolution_problem(int(1.5 * n), n, 8.0, 32, 1e-6, 1e-6, 1e-4, seed)


def batch_c3(seed=2, count=512, nmin=256, nmax=65536, nlambda=16):
    """512 real problems, n log-uniform in [nmin, nmax], m = n + U[0, n/2], sigma ~ U[2, 16],
    lambda path log-spaced 1e-6 .. 1."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        m = n + int(rng.integers(0, n // 2 + 1))
        sigma = float(rng.uniform(2.0, 16.0))
        probs.append(deconvolution_problem(m, n, sigma, int(math.ceil(4 * sigma)), 1e-6, 1e-6, 1.0,
                                           int(rng.integers(1 << 30))))
    lams = np.logspace(-6, 0, nlambda)
    return probs, lams


def paper_problem(n, seed=0):
    """Sec. 7.1: complex standard-normal square T, known x, y = (T^H T + lam I) x, lam = sqrt(2n)."""
    rng = np.random.default_rng(seed)
    col = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    row = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    row[0] = col[0]
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = math.sqrt(2 * n)
    return dict(col=col, row=row, x_true=x, lam=lam, m=n, n=n)


def random_problem(m, n, lam, seed, complex_data=True):
    """Small dense-checkable problem with standard-normal generator and data."""
    rng = np.random.default_rng(seed)
    if complex_data:
        col = rng.standard_normal(m) + 1j * rng.standard_normal(m)
        row = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    else:
        col = rng.standard_normal(m)
        row = rng.standard_normal(n)
        b = rng.standard_normal(m)
    row[0] = col[0]
    return dict(col=col, row=row, b=b, lam=lam, m=m, n=n)


def general_problem(m, n, p, seed, complex_data=False):
    """Sec. 7.1's general problem: T (m x n) and L (p x n) Toeplitz with standard-normal generators, x_true
    standard normal, b = T x_true; the system is (T^H T + L^H L) x = T^H b.  Returns dict(col, row, lcol,
    lrow, b, x_true, m, n, p)."""
    rng = np.random.default_rng(seed)
    draw = (lambda k: rng.standard_normal(k) + 1j * rng.standard_normal(k)) if complex_data else rng.standard_normal
    col, row, lcol, lrow, x_true = draw(m), draw(n), draw(p), draw(n), draw(n)
    row[0] = col[0]
    lrow[0] = lcol[0]
    b = toeplitz_matvec(col, row, x_true)
    return dict(col=col, row=row, lcol=lcol, lrow=lrow, b=b, x_true=x_true, m=m, n=n, p=p)


def nufft_problem(n=4096, K=4096, seed=6, l_scale=1e-2):
    """Sec. 7.4's reconstruction workload: a length-n signal of three sinusoids with random frequencies in
    [0, 0.02]; K spectral samples X_k = sum_s x_s exp(-2 pi i f_k s) at frequencies drawn from the triangular
    distribution on [-1/2, 1/2); Voronoi-cell density weights w_k (half the distance between the neighbours
    on the unit circle of frequencies, summing to 1); L = l_scale x [-1, 2, -1], a square second difference.
    Returns dict(f, w, X, x_true, lcol, lrow)."""
    rng = np.random.default_rng(seed)
    s = np.arange(n)
    fr = rng.uniform(0.0, 0.02, 3)
    amp = rng.standard_normal(3)
    ph = rng.uniform(0.0, 2 * np.pi, 3)
    x_true = sum(a * np.cos(2 * np.pi * fq * s + p) for a, fq, p in zip(amp, fr, ph))
    f = np.sort(rng.triangular(-0.5, 0.0, 0.5, K))
    fp = np.concatenate([[f[-1] - 1.0], f, [f[0] + 1.0]])
    w = (fp[2:] - fp[:-2]) / 2
    X = np.exp(-2j * np.pi * np.outer(f, s)) @ x_true
    lcol = np.zeros(n)
    lcol[:2] = [2 * l_scale, -l_scale]
    return dict(f=f, w=w, X=X, x_true=x_true, lcol=lcol, lrow=lcol.copy(), n=n, K=K)

