"""The library's host set-up (Sec. 2 1D matrices, Appendix line solves) on
the CPU: its mass and stiffness bands against the oracle's 1D matrices, its
pivot-free band LU against M + d K, and its partition tables (fundamental
solutions and transfer matrices of the segment-parallel substitution, for
32-, 33- and 44-row segments) against plain banded substitution.

tests/host/setup1d_check.cpp is compiled with the library's own
csrc/setup1d.cpp (plain C++, no CUDA) and prints what is compared here."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as ora

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_08158_gb300", "csrc")

CASES = [(128, 3, False), (128, 2, False), (100, 2, False), (96, 3, True), (40, 4, False), (300, 2, True),
         (5, 1, False), (33, 2, False)]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("host") / "setup1d_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host", "setup1d_check.cpp"),
                    os.path.join(CSRC, "setup1d.cpp"), "-o", exe], check=True, capture_output=True)
    return exe


def _run(exe, ne, p, natural, d, seg):
    out = subprocess.run([exe, str(ne), str(p), str(int(natural)), repr(d), str(seg)], check=True,
                         capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "band":
            m, w = int(f[2]), int(f[3])
            res[f[1]] = np.array([float(v) for v in f[4:]]).reshape(m, w)
        elif f[0] == "lohi":
            res["lohi"] = (int(f[1]), int(f[2]))
        else:
            res[f[0]] = float(f[1])
    return res


def _dense(band):
    m, w = band.shape
    p = w // 2
    A = np.zeros((m, m))
    for i in range(m):
        for k in range(-p, p + 1):
            if 0 <= i + k < m:
                A[i, i + k] = band[i, k + p]
            else:
                assert band[i, k + p] == 0.0   # entries outside the matrix are stored as zeros
    return A


@pytest.mark.parametrize("ne,p,natural", CASES)
def test_bands_match_oracle_and_toeplitz_rows_are_exact(checker, ne, p, natural):
    r = _run(checker, ne, p, natural, 1e-4, 32)
    s = ora.Space((ne, 2, 2), p, natural=natural)
    for which in ("M", "K"):
        ref = s.mat(0, which)
        got = _dense(r[which])
        assert got.shape == ref.shape
        # Toeplitz rows are set to one exact stencil row (within 1e-12 of the row)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), which
        lo, hi = r["lohi"]
        if hi > lo:
            band = r[which]
            mid = (lo + hi) // 2
            assert np.array_equal(band[lo:hi], np.repeat(band[mid:mid + 1], hi - lo, axis=0)), which


@pytest.mark.parametrize("ne,p,natural", CASES)
@pytest.mark.parametrize("d", [1e-6, 1e-3, 0.25])
def test_band_lu_reproduces_operator(checker, ne, p, natural, d):
    assert _run(checker, ne, p, natural, d, 32)["lu_resid"] <= 1e-14


@pytest.mark.parametrize("ne,p,natural", CASES)
@pytest.mark.parametrize("seg", [32, 33, 44])
def test_partitioned_solve_equals_plain_substitution(checker, ne, p, natural, seg):
    m = ne + p - (0 if natural else 2)
    r = _run(checker, ne, p, natural, 1e-5, seg)
    assert r["segments"] == -(-m // seg)
    assert r["part_err"] <= 1e-13


def _choose_seg():
    """The library's segment-length rule (internal C++ symbol ads::choose_seg)."""
    import ctypes
    from paper_1911_08158_gb300 import library
    f = getattr(library(), "_ZN3ads10choose_segEPKii")
    f.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    f.restype = ctypes.c_int
    return lambda m, elem: f((ctypes.c_int * 3)(*m), elem)


@pytest.mark.parametrize("m,elem,seg", [
    ((128, 128, 128), 4, 32),      # 4 line groups x 4 segments: one round of 16 warps
    ((129, 129, 129), 4, 44),      # 5 groups: 3 segments of 44 rows fit one round, 4 of 33 do not
    ((129, 129, 129), 8, 33),      # FP64 CTA of 8 warps: 44 rows save no round
    ((97, 130, 5), 4, 33),         # 32 s + 1 unknowns: one segment fewer with 33 rows
    ((130, 129, 3), 4, 44),
    ((176, 176, 176), 4, 44),      # 6 groups: 4 segments of 44 (2 rounds) vs 6 of 32 (3 rounds)
    ((70, 70, 70), 8, 44),         # FP64: 2 segments of 44 (one round) vs 3 of 32 (two)
    ((300, 4, 3), 8, 44),          # 7 segments of 44 rows: the 256-thread FP64 CTA
    ((400, 300, 10), 8, 32),       # more than 8 segments of 44: K1 has no wide 44-row CTA
    ((265, 360, 10), 4, 33),       # 9 segments of 44 along y: excluded; 33 rows save a segment over 32
    ((512, 4, 4), 4, 32),
])
def test_segment_length_choice(m, elem, seg):
    assert _choose_seg()(m, elem) == seg


def test_segment_length_never_exceeds_what_k1_instantiates():
    """44-row segments only while every line takes at most 8 of them (the
    single-CTA layout, also in FP64), for all axis lengths up to 512."""
    choose = _choose_seg()
    for a in range(1, 513, 3):
        for b in range(1, 513, 5):
            for elem in (4, 8):
                if choose((a, b, 17), elem) == 44:
                    assert -(-a // 44) <= 8 and -(-b // 44) <= 8, (a, b, elem)
