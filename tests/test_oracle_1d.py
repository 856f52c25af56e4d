"""Pins of the oracle's 1D pieces (Sec. 2 and the Appendix) against things
fixed independently of it: NumPy's Gauss rule, SciPy's B-spline evaluator,
polynomial exactness, closed-form cardinal B-spline stencils, partition of
unity and the row-sum identities."""
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import oracle as ora
from tests import splines_ref as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cardinal_stencils.txt")


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_matches_numpy_and_is_exact(q):
    x, w = ora.gauss(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(x, xr, atol=1e-15)
    np.testing.assert_allclose(w, wr, atol=1e-15)
    # exact for all polynomials up to degree 2q-1
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # and not for degree 2q
    assert abs(np.sum(w * x ** (2 * q)) - 2.0 / (2 * q + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_matches_scipy_and_partition_of_unity(p):
    ne = 7
    fs, t = ref.basis_funcs(ne, p)
    rng = np.random.default_rng(p)
    for e in range(ne):
        for x in rng.uniform(e / ne, (e + 1) / ne, size=3):
            N, dN = ora.basis(ne, p, p + e, x)
            Nr = np.array([np.nan_to_num(f(x)) for f in fs])
            dNr = np.array([np.nan_to_num(f.derivative()(x)) for f in fs])
            np.testing.assert_allclose(N, Nr, atol=1e-14)
            np.testing.assert_allclose(dN, dNr, atol=1e-11)
            assert abs(N.sum() - 1.0) < 1e-14          # partition of unity
            assert abs(dN.sum()) < 1e-11                # its derivative
            assert np.all(N >= -1e-15)
            # local support: only e .. e+p are nonzero
            nz = np.nonzero(np.abs(N) > 0)[0]
            assert nz.min() >= e and nz.max() <= e + p


def test_knot_vector_open_uniform():
    t = ora.knots(5, 3, 2.0)
    np.testing.assert_allclose(t, [0, 0, 0, 0, 0.4, 0.8, 1.2, 1.6, 2, 2, 2, 2])


def _cardinal(m, x, d=0):
    s = Fraction(0)
    for j in range(m + 2):
        y = x - j
        if y > 0:
            s += (-1) ** j * comb(m + 1, j) * Fraction(y) ** (m - d)
    return s / factorial(m - d)


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        p, kind, nums, den = int(f[0]), f[1], [int(v) for v in f[2:-1]], int(f[-1])
        rows[(p, kind)] = [Fraction(v, den) for v in nums]
    return rows


def test_golden_stencils_are_the_closed_form():
    for (p, kind), vals in _golden().items():
        if kind == "mass":
            cf = [_cardinal(2 * p + 1, p + 1 + k) for k in range(-p, p + 1)]
        else:
            cf = [-_cardinal(2 * p + 1, p + 1 + k, 2) for k in range(-p, p + 1)]
        assert cf == vals, (p, kind)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_interior_rows_match_cardinal_stencils(p):
    ne, L = 4 * p + 6, 1.7
    h = L / ne
    M, K, B = ora.mats1d(ne, p, L)
    mass = np.array([float(_cardinal(2 * p + 1, p + 1 + k)) for k in range(-p, p + 1)])
    stiff = np.array([float(-_cardinal(2 * p + 1, p + 1 + k, 2)) for k in range(-p, p + 1)])
    # rows whose support (and neighbours' support) avoids the repeated end knots
    for i in range(2 * p, ne + p - 2 * p):
        np.testing.assert_allclose(M[i, i - p:i + p + 1], h * mass, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(K[i, i - p:i + p + 1], stiff / h, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p,ne", [(1, 5), (2, 6), (3, 7), (4, 9), (2, 1), (3, 2)])
def test_mats_match_scipy_assembly(p, ne):
    M, K, B = ora.mats1d(ne, p, 1.0)
    Mr, Kr, Br = ref.mats(ne, p, 1.0)
    np.testing.assert_allclose(M, Mr, atol=1e-15)
    np.testing.assert_allclose(K, Kr, atol=1e-11)
    np.testing.assert_allclose(B, Br, atol=1e-12)


@pytest.mark.parametrize("p,ne", [(1, 4), (2, 6), (3, 8), (4, 9)])
def test_row_sums_band_and_symmetry(p, ne):
    L = 1.3
    M, K, B = ora.mats1d(ne, p, L)
    n = ne + p
    t = ora.knots(ne, p, L)
    # sum_j M_ij = int N_i = (t_{i+p+1} - t_i)/(p+1)
    np.testing.assert_allclose(M.sum(1), (t[p + 1:p + 1 + n] - t[:n]) / (p + 1), atol=1e-15)
    # K annihilates constants (sum of N_j = 1)
    np.testing.assert_allclose(K.sum(1), 0.0, atol=1e-12)
    # sum_c B[a,c] = int N'_a = N_a(L) - N_a(0)
    e = np.zeros(n); e[0] = -1.0; e[-1] = 1.0
    np.testing.assert_allclose(B.sum(1), e, atol=1e-13)
    # B + B^T = [N_a N_c]_0^L
    bt = np.zeros((n, n)); bt[0, 0] = -1.0; bt[-1, -1] = 1.0
    np.testing.assert_allclose(B + B.T, bt, atol=1e-13)
    # banded: M_ij = 0 iff |i-j| > p (Appendix)
    i, j = np.indices((n, n))
    assert np.all(M[np.abs(i - j) > p] == 0.0) and np.all(K[np.abs(i - j) > p] == 0.0)
    assert np.all(M[np.abs(i - j) <= p] > 0.0)
    np.testing.assert_allclose(M, M.T, atol=0)
    np.testing.assert_allclose(K, K.T, atol=1e-15)


def test_restricted_matrices_spd():
    s = ora.Space((5, 6, 4), 3, (1.0, 2.0, 0.5))
    for a in range(3):
        for w in "MK":
            A = s.mat(a, w)
            assert np.linalg.eigvalsh(A).min() > 0


def test_ricker_closed_form():
    f, t0 = 8.0, 0.125
    assert ora.ricker(f, t0, t0) == 1.0
    tz = t0 + 1.0 / (np.pi * f * np.sqrt(2.0))        # zero crossing
    assert abs(ora.ricker(f, t0, tz)) < 1e-15
    t = 0.3
    a = (np.pi * f * (t - t0)) ** 2
    assert abs(ora.ricker(f, t0, t) - (1 - 2 * a) * np.exp(-a)) < 1e-16


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_l2_projection_converges_at_order_p_plus_1(p):
    """Spatial order (soft pin; the paper states no rate): the L2 projection of
    a smooth function onto the degree-p spline space of ne uniform elements
    has an L2 error O(h^(p+1)), the textbook rate of the space that the
    oracle's basis, quadrature and mass matrix span together.  Observed
    log2 error ratios between ne = 12, 24, 48 must lie within 0.25 of p + 1
    (measured: 2.03 2.01 | 3.03 3.00 | 4.12 4.03 | 5.14 5.03)."""
    f = lambda x: np.sin(2 * np.pi * x) + x * x
    gx, gw = np.polynomial.legendre.leggauss(p + 6)   # exact enough for f N_i and the error integral

    def proj_error(ne):
        n = ne + p
        M = ora.mats1d(ne, p)[0]
        b = np.zeros(n)
        pts = []
        for e in range(ne):
            a, h = e / ne, 1.0 / ne
            for xg, wg in zip(gx, gw):
                x, w = a + 0.5 * h * (xg + 1), 0.5 * h * wg
                N, _ = ora.basis(ne, p, p + e, x)
                b += w * f(x) * N
                pts.append((x, w, N))
        c = np.linalg.solve(M, b)
        return np.sqrt(sum(w * (f(x) - N @ c) ** 2 for x, w, N in pts))

    errs = [proj_error(ne) for ne in (12, 24, 48)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for r in rates:
        assert abs(r - (p + 1)) < 0.25, (p, errs, rates)
