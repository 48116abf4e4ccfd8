"""The C-ABI library builds, loads and exports every entry point include/tikh.h declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tikh.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(tikh_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    from paper_1302_6945_gb300 import build as B
    from paper_1302_6945_gb300 import tikh
    B.build()
    L = tikh.lib()
    names = declared()
    assert len(names) >= 8
    for name in names:
        assert hasattr(L, name), name
    assert set(tikh.EXPORTED) <= set(names)


def test_strerror_and_invalid_plan_without_gpu():
    from paper_1302_6945_gb300 import tikh
    assert tikh.tikh_strerror(tikh.TIKH_EINVAL) == "invalid argument"
    with pytest.raises(tikh.TikhError):
        tikh.tikh_plan_create(0, 4)



@pytest.mark.parametrize("field,value", [("n_lim", 3), ("n_lim", 65), ("m_min", 33), ("fill", 2), ("eps_diff", -1.0),
                                         ("max_difficult", 0), ("refine_steps", 9), ("batch", 0), ("graph", 2),
                                         ("prod_direct_max", -1), ("prod_direct_max", 4097),
                                         ("eval_direct_max", -1), ("eval_direct_max", 4097), ("wait_polls", -1),
                                         ("wait_polls", (1 << 30) + 1), ("refine_tol", -1.0),
                                         ("fft_radix", 2), ("fft_tile", 300), ("fft_tile", 8192)])
def test_invalid_options_are_rejected_before_any_device_work(field, value):
    # argument checks come first, so they hold on a machine without a GPU
    from paper_1302_6945_gb300 import tikh
    o = tikh.tikh_opts(32, 0, 0, 1e-8, 4096, 0, 1, 0, 0, 0, 0, 0.0)
    setattr(o, field, value)
    with pytest.raises(tikh.TikhError) as e:
        tikh.tikh_plan_create(64, 64, tikh.TIKH_R64, tikh.TIKH_PREC_FP64, o)
    assert "invalid" in str(e.value).lower() or str(tikh.TIKH_EINVAL) in str(e.value)
