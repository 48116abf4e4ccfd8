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


@pytest.mark.parametrize("m,n,pl,dtype,n_lim", [(0, 8, 8, 0, 30), (8, 0, 8, 0, 30), (8, 8, 0, 0, 30),
                                                (8, 8, 8, 7, 30), (40, 30, 20, 0, 64), (40, 30, 20, 0, 2)])
def test_general_plan_arguments_are_checked_before_any_device_work(m, n, pl, dtype, n_lim):
    # sizes, dtype and a leaf above 42 conditions (3 M > 42 for the 7 x 7 basis) are refused on the host
    from paper_1302_6945_gb300 import tikh
    o = tikh.tikh_opts(n_lim, 0, 0, 1e-12, 4096, 0, 1, 0, 0, 0, 0, 0.0)
    with pytest.raises(tikh.TikhError) as e:
        tikh.tikh_plan_create_general(m, n, pl, dtype, o)
    assert e.value.status == tikh.TIKH_EINVAL


def test_general_solves_refuse_a_missing_plan():
    from paper_1302_6945_gb300 import tikh
    for f in (tikh.tikh_solve_general, tikh.tikh_solve_general_normal):
        with pytest.raises(tikh.TikhError) as e:
            f(None, 1, 1, 1, 1, 1, 1)
        assert e.value.status == tikh.TIKH_EINVAL
    with pytest.raises(tikh.TikhError):
        tikh.tikh_solve_general_strided(None, 1, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0)


def test_inverse_entry_points_refuse_a_missing_handle():
    # host checks before any device work: a null plan or handle is TIKH_EINVAL, destroy(NULL) is a no-op
    from paper_1302_6945_gb300 import tikh
    with pytest.raises(tikh.TikhError) as e:
        tikh.tikh_inverse_create(None, 1, 1, 1.0, 4)
    assert e.value.status == tikh.TIKH_EINVAL
    with pytest.raises(tikh.TikhError) as e:
        tikh.tikh_inverse_apply(None, 1, 1, 0, 1, 0, 0, 0)
    assert e.value.status == tikh.TIKH_EINVAL
    with pytest.raises(tikh.TikhError):
        tikh.tikh_inverse_generators(None, 1)
    with pytest.raises(tikh.TikhError):
        tikh.tikh_inverse_info(None)
    tikh.tikh_inverse_destroy(None)
