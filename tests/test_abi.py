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

