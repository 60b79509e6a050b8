"""The C-ABI library loads on any host and exports every entry point that
include/lfsr.h declares (no compute call: no GPU is needed)."""
import os
import re

from paper_2206_05047_gb300 import lfsr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char \*)\s*(lfsr_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2206_05047_gb300 import build
    build.build()
    lib = lfsr.load_library()
    declared = _declared()
    assert declared == set(lfsr.EXPORTS)
    for name in declared:
        assert getattr(lib, name) is not None


def test_struct_layouts_match_header():
    import ctypes as C
    # lfsr_params: 7 int32 + 2 pointers + 3 doubles + 2 int32 + double + int32 + double + int32
    assert C.sizeof(lfsr.lfsr_params) == 112
    assert C.sizeof(lfsr.lfsr_stats_t) == 4 * 4 + 8 * 2 + 8 * 2 + 8 * 8 + 8 * 8


def test_invalid_arguments_fail_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(2, 3, 8, 8, 2, blur, np.zeros((16, 16), np.float32))
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "odd" in lfsr.last_error(None)
