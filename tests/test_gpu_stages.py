"""Stage-wise parity through the C-ABI test hooks: the FFT engine and one leaf, on identical inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1302_6945_gb300 import tikh

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 12, 40, 49, 64, 125, 343, 640, 2048, 4096, 4200, 20480,
                               163840, 327680 * 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_fft_matches_definition(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = tikh.fft(torch.tensor(x, device=DEV), sign).cpu().numpy()
    ref = np.fft.ifft(x) * n if sign > 0 else np.fft.fft(x)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 1e-14 * max(1.0, np.log2(n)) * 4, err


def _leaf_case(K, seed, zero_frac=0.3):
    rng = np.random.default_rng(seed)
    e = rng.permutation(4 * K)[:K]
    sigma = np.exp(2j * np.pi * e / (4 * K))
    r = rng.standard_normal((K, 5)) + 1j * rng.standard_normal((K, 5))
    r[rng.random((K, 5)) < zero_frac] = 0.0
    r[:, 4] *= 0.1
    return sigma, r


@pytest.mark.parametrize("K,seed", [(1, 0), (4, 1), (8, 2), (20, 3), (32, 4), (40, 5), (64, 6)])
def test_leaf_matches_oracle_leaf(K, seed):
    sigma, r = _leaf_case(K, seed)
    delta = [-7, -9, -9, -8, 0]
    g = tikh.leaf(torch.tensor(sigma, device=DEV), torch.tensor(r, device=DEV), delta, eps=1e-8)
    o = oracle.leaf(sigma, r.copy(), delta, eps=1e-8)
    # decisions are unique here (no ties): identical order, pivots, degrees, deferrals
    assert list(g["order"]) == list(o["order"])
    assert list(g["pivot"]) == list(o["pivot"])
    assert list(g["delta"]) == list(o["delta"])
    assert g["deferred"] == sorted(o["deferred"])
    # the basis entrywise (the device trims to the degree bounds; beyond them the oracle has zeros)
    for E in range(25):
        lg = g["len"][E]
        a = g["B"][E, :lg]
        b = o["B"][E, :lg]
        assert np.abs(o["B"][E, lg:]).max(initial=0.0) == 0.0
        scale = max(np.abs(o["B"][E]).max(initial=0.0), 1e-300)
        assert np.abs(a - b).max(initial=0.0) <= 1e-12 * scale, E


def test_leaf_deferral_matches_oracle():
    sigma, r = _leaf_case(32, 11, zero_frac=0.6)
    for eps in (0.1, 0.3, 0.6):
        g = tikh.leaf(torch.tensor(sigma, device=DEV), torch.tensor(r, device=DEV), [-3, -3, -3, -3, 0], eps=eps)
        o = oracle.leaf(sigma, r.copy(), [-3, -3, -3, -3, 0], eps=eps)
        assert g["deferred"] == sorted(o["deferred"]), eps
        assert list(g["order"]) == list(o["order"])


def test_leaf_series_reciprocal_is_within_fp64_rounding():
    # the leaf's 1/|r_pi|^2: FP32 seed + one third-order series step; over the whole exponent range it
    # admits (biased exponent 3 .. 2043) and random mantissas it must be within 1 ulp of the correctly
    # rounded 1/d (the series' truncation e^3 < 2^-63 leaves only the final roundings)
    import ctypes
    rng = np.random.default_rng(17)
    mant = 1.0 + rng.random(200000)
    expo = rng.integers(-1018, 1018, 200000)
    d = np.ldexp(mant, expo)
    d = np.concatenate([d, [1.0, 2.0, 1.5, np.nextafter(2.0, 0.0), np.ldexp(1.0, -1018), np.ldexp(1.0, 1017)]])
    x = torch.tensor(d, dtype=torch.float64, device=DEV)
    out = torch.empty_like(x)
    tikh.tikh_test_rcp(x.numel(), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                       torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    ref = 1.0 / d
    ulp = np.abs(np.spacing(ref))
    assert (np.abs(got - ref) <= ulp).all(), np.max(np.abs(got - ref) / ulp)


def test_column_scaling_by_exponent_arithmetic_matches_the_multiply():
    # the products' loaders scale basis coefficients by the column's power of two through the exponent field;
    # over normal, sub-normal, zero, huge, infinite and NaN values and column maxima from sub-normal to huge it
    # must give exactly what the FP64 multiply by the same power of two gives
    import ctypes
    rng = np.random.default_rng(23)
    n = 200000
    with np.errstate(over="ignore"):
        v = np.ldexp(rng.standard_normal(n), rng.integers(-1074, 1023, n))
        mx = np.abs(np.ldexp(1.0 + rng.random(n), rng.integers(-1074, 1023, n)))
    v[:8] = [0.0, -0.0, 5e-324, -1e-310, np.inf, -np.inf, 1.7e308, -2.2250738585072014e-308]
    mx[:16] = [0.0, 5e-324, 1e-310, 2.2250738585072014e-308, 1.0, 0.75, 1.7e308, np.inf, 0.5, 1e-300, 1e300,
               4.0, 3.9e-308, 8.9e307, 1.1e-308, 2.0]
    vv = torch.tensor(np.append(v, np.nan), dtype=torch.float64, device=DEV)
    bits = torch.tensor(np.append(mx, 1.0).view(np.int64), dtype=torch.int64, device=DEV)
    oe, om = torch.empty_like(vv), torch.empty_like(vv)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    tikh.tikh_test_scale(vv.numel(), p(vv), p(bits), p(oe), p(om), torch.cuda.current_stream().cuda_stream)
    a, b = oe.cpu().numpy(), om.cpu().numpy()
    assert np.array_equal(a.view(np.int64)[:-1], b.view(np.int64)[:-1])
    assert np.isnan(a[-1]) and np.isnan(b[-1])


@pytest.mark.parametrize("K,delta_in,seed", [(8, [-10, -10, 0, 0, 0], 1), (12, [-30, -9, -9, -30, 0], 2),
                                             (6, [-4, -20, -4, -4, -4], 3)])
def test_leaf_rows_of_unpivoted_columns_are_exact_identity_rows(K, delta_in, seed):
    # the evaluations and products skip the rows of a basis outside the columns pivoted in its node and use
    # them as identity rows: the leaf kernel must produce them exactly (same pivots as the oracle's leaf)
    rng = np.random.default_rng(seed)
    sigma = np.exp(2j * np.pi * rng.permutation(4 * K)[:K] / (4 * K))
    phi = rng.standard_normal((K, 5)) + 1j * rng.standard_normal((K, 5))
    g = tikh.leaf(torch.tensor(sigma, device=DEV), torch.tensor(phi, device=DEV), delta_in, eps=1e-12)
    o = oracle.leaf(sigma, phi.copy(), delta_in, eps=1e-12)
    assert list(g["pivot"][:K]) == list(o["pivot"][:K])
    unpivoted = [i for i in range(5) if i not in set(int(p) for p in g["pivot"][:K])]
    assert unpivoted
    B, ln = g["B"], g["len"]
    for i in unpivoted:
        for j in range(5):
            e = B[5 * i + j, :ln[5 * i + j]]
            if j == i:
                assert ln[5 * i + j] >= 1 and e[0] == 1.0 and not np.any(e[1:])
            else:
                assert not np.any(e)
