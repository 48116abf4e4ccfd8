"""The allocation-free DFT entry point (tikh_fft_noalloc) against the allocating one (tikh_test_fft).

Some callers cannot allocate device memory during a call (their device memory belongs to another
allocator or a fixed budget, or their inner loop cannot afford an allocation); tikh_fft_noalloc
serves them from a fixed device array.  This file runs last so that
a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1302_6945_gb300 import tikh

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(fn, x, sign):
    y = x.clone()
    fn(y.numel(), ctypes.c_void_p(y.data_ptr()), sign, torch.cuda.current_stream().cuda_stream)
    return y.cpu().numpy()


@pytest.mark.parametrize("n", [7, 40, 4096, 5000, 65536])
def test_noalloc_matches_allocating_entry_point_twice(n):
    rng = np.random.default_rng(n)
    for call in range(2):  # two calls in a row share (and rewrite) the same scratch
        sign = 1 if call == 0 else -1
        x = torch.tensor(rng.standard_normal(n) + 1j * rng.standard_normal(n), device=DEV)
        ref = _run(tikh.tikh_test_fft, x, sign)
        got = _run(tikh.tikh_fft_noalloc, x, sign)
        assert np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), (n, call)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros(65536 * 2, dtype=torch.complex128, device=DEV)
    with pytest.raises(tikh.TikhError):
        tikh.tikh_fft_noalloc(x.numel(), ctypes.c_void_p(x.data_ptr()), 1, torch.cuda.current_stream().cuda_stream)
