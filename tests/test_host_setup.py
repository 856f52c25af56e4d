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
