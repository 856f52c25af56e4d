"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ads.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ads_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1911_08158_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_and_launch_count_without_gpu():
    import paper_1911_08158_gb300 as ads
    L = ads.library()
    assert L.ads_launch_count() >= 0
    assert isinstance(L.ads_last_error(), bytes)


def test_invalid_arguments_rejected_on_host():
    import paper_1911_08158_gb300 as ads
    # p out of range is rejected before any device call
    with pytest.raises(ads.AdsError) as e:
        ads.Simulation(4, 7, 0.01, use_torch=False)
    assert e.value.code == -5
    with pytest.raises(ads.AdsError) as e:
        ads.Simulation(4, 2, -1.0, use_torch=False)
    assert e.value.code == -1
    with pytest.raises(ads.AdsError) as e:
        ads.Simulation((4, 0, 4), 2, 0.01, use_torch=False)
    assert e.value.code == -1
    # measurement calls validate their arguments before touching the device
    L = ads.library()
    ms = ctypes.c_float()
    assert L.ads_profile_rhs(None, 5, ctypes.byref(ms)) == -1
    assert L.ads_profile_rhs(None, 5, None) == -1


def test_estimate_bytes_is_host_only_and_consistent():
    from paper_1911_08158_gb300 import estimate_bytes
    w32 = estimate_bytes((32, 40, 24), 2, "wave", "fp32")
    w64 = estimate_bytes((32, 40, 24), 2, "wave", "fp64")
    e32 = estimate_bytes((32, 40, 24), 2, "elastic", "fp32")
    big = estimate_bytes((64, 40, 24), 2, "wave", "fp32")
    assert 0 < w32 < w64 and w32 < e32 and w32 < big
    # the four state arrays alone: (34 padded to 40) x 40 x 24 x 4 bytes each
    assert w32 >= 4 * 40 * 40 * 24 * 4
    assert estimate_bytes((32, 40, 24), 9, "wave", "fp32") == 0
    assert estimate_bytes((0, 40, 24), 2, "wave", "fp32") == 0
