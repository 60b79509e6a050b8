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
            names |= set(re.findall(r"^\s*(?:int64_t|int|void|const char \*)\s*(lfsr_\w+)\s*\(", src, re.M))
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
    # + views pointer + int32 + weights int32 + 4 floats + proj_err pointer
    # + disparity_views pointer + adjoint int32 (padded)
    assert C.sizeof(lfsr.lfsr_params) == 168
    assert lfsr.lfsr_params.weights.offset == 124 and lfsr.lfsr_params.proj_err.offset == 144
    assert lfsr.lfsr_params.disparity_views.offset == 152 and lfsr.lfsr_params.adjoint.offset == 160
    assert C.sizeof(lfsr.lfsr_stats_t) == 4 * 4 + 8 * 2 + 8 * 2 + 8 * 8 + 8 * 8 + 8 * 2


def test_invalid_arguments_fail_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(2, 3, 8, 8, 2, blur, np.zeros((16, 16), np.float32))
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "odd" in lfsr.last_error(None)


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "lfsr.h")).read()
    defs = dict(re.findall(r"^#define\s+(LFSR_\w+)\s+\(?(-?[0-9.]+)\)?", src, re.M))
    for name, val in defs.items():
        if hasattr(lfsr, name):
            assert float(getattr(lfsr, name)) == float(val), name
    for name in ("LFSR_FP32", "LFSR_FP16_STORAGE", "LFSR_BF16_STORAGE", "LFSR_FP16_MAX_INV_MU",
                 "LFSR_KEEP_VIEWS_FP32", "LFSR_WEIGHTS_PATCH", "LFSR_WEIGHTS_PAPER",
                 "LFSR_ADJOINT_EXACT", "LFSR_ADJOINT_BACKWARD_WARP",
                 "LFSR_EINVAL", "LFSR_EUNSUPPORTED", "LFSR_MEM_DEVICE"):
        assert name in defs and hasattr(lfsr, name), name


def test_precision_is_validated_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    for bad in (3, lfsr.LFSR_KEEP_VIEWS_FP32 | 3, 512):
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.create(3, 3, 8, 8, 2, blur, disp, precision=bad)
        assert e.value.code == lfsr.LFSR_EINVAL
    # half storage cannot hold duals bounded by 1/mu = 1e4
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(3, 3, 8, 8, 2, blur, disp, mu=1e-4, precision=lfsr.LFSR_FP16_STORAGE)
    assert e.value.code == lfsr.LFSR_EUNSUPPORTED
    assert "8192" in lfsr.last_error(None)


def test_batch_arguments_are_validated_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    job = dict(U=3, V=3, H=8, W=8, scale=2, blur=blur, disparity=disp)
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.Batch([])
    assert e.value.code == lfsr.LFSR_EINVAL
    # light fields of one batch share the solver constants
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.Batch([job, dict(job, mu=2.0)])
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "share" in lfsr.batch_last_error(None)


def test_view_subsets_are_validated_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    for bad in ([3, 1], [0, 9], [-1, 2], []):
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.create(3, 3, 8, 8, 2, blur, disp, views=bad)
        assert e.value.code == lfsr.LFSR_EINVAL
    base = lfsr.estimate_state_bytes(U=5, V=5, H=32, W=32, scale=2, blur=blur,
                                     disparity=np.zeros((64, 64), np.float32))
    star = lfsr.estimate_state_bytes(U=5, V=5, H=32, W=32, scale=2, blur=blur,
                                     disparity=np.zeros((64, 64), np.float32),
                                     views=[2, 6, 7, 8, 10, 11, 12, 13, 14, 16, 17, 18, 22])
    assert star < base


def test_weight_scheme_is_validated_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    bad = [dict(weights=2), dict(weights=-1), dict(weights="paper", sigma_s=-1.0),
           dict(weights="paper", sigma_e=float("nan")), dict(weights="paper", sigma_o1=float("inf")),
           dict(weights="paper", sigma_o2=-0.5),
           dict(weights="paper", sigma_o2=1.0, proj_err=np.full((16, 16), np.nan, np.float32))]
    for kw in bad:
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.create(3, 3, 8, 8, 2, blur, disp, **kw)
        assert e.value.code == lfsr.LFSR_EINVAL, kw
    with pytest.raises(ValueError):
        lfsr.create(3, 3, 8, 8, 2, blur, disp, weights="paper", proj_err=np.zeros(5))
    # the occlusion factor is one more HR float map
    kw = dict(U=5, V=5, H=32, W=32, scale=2, blur=blur, disparity=np.zeros((64, 64), np.float32))
    assert (lfsr.estimate_state_bytes(weights="paper", **kw) -
            lfsr.estimate_state_bytes(**kw)) == 4 * 64 * 64
    # a batch shares the scheme and its sigmas
    job = dict(U=3, V=3, H=8, W=8, scale=2, blur=blur, disparity=disp, weights="paper",
               sigma_s=8.0)
    for other in (dict(job, weights="patch"), dict(job, sigma_s=4.0)):
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.Batch([job, other])
        assert e.value.code == lfsr.LFSR_EINVAL
        assert "weight scheme" in lfsr.batch_last_error(None)


def test_warp_options_are_validated_without_gpu():
    import numpy as np
    import pytest
    blur = np.ones((3, 3), np.float32) / 9
    disp = np.zeros((16, 16), np.float32)
    for bad in (2, -1):
        with pytest.raises(lfsr.LfsrError) as e:
            lfsr.create(3, 3, 8, 8, 2, blur, disp, adjoint=bad)
        assert e.value.code == lfsr.LFSR_EINVAL
    maps = np.zeros((9, 16, 16), np.float32)
    maps[4, 3, 3] = np.inf
    with pytest.raises(lfsr.LfsrError) as e:
        lfsr.create(3, 3, 8, 8, 2, blur, disp, disparity_views=maps)
    assert e.value.code == lfsr.LFSR_EINVAL
    assert "disparity_views" in lfsr.last_error(None)
    with pytest.raises(ValueError):
        lfsr.create(3, 3, 8, 8, 2, blur, disp, disparity_views=np.zeros((8, 16, 16)))
    # a subset of views takes one map per listed view
    with pytest.raises(ValueError):
        lfsr.create(3, 3, 8, 8, 2, blur, disp, views=[1, 4, 7], disparity_views=maps)
    kw = dict(U=3, V=3, H=8, W=8, scale=2, blur=blur, disparity=disp)
    base = lfsr.estimate_state_bytes(**kw)
    assert lfsr.estimate_state_bytes(disparity_views=np.zeros((9, 16, 16)), **kw) - base == 4 * 9 * 256
    assert lfsr.estimate_state_bytes(adjoint="backward", **kw) - base == 4 * 9 * 64
