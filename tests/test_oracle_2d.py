"""Pins of the oracle's 2D problems (n_elem[2] = 0: one constant function
along z), the setting in which Sec. 2 and Sec. 3 derive the method.

- the split step against a dense 2D solve built from SciPy's B-splines;
- the 2D load vector of a Gaussian against SciPy 1D loads;
- the Sec. 3 eigenmode recurrence in 2D: a product of 1D generalised
  eigenvectors stays a mode, its amplitude following Newmark on
  m~ = (1 + eta lx)(1 + eta ly) - eta (lx + ly),  k = lx + ly;
- plane-strain elasticity against a direct 2D quadrature of the bilinear
  form, the z component decoupled.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as ora
from tests import splines_ref as ref


def test_space_shape_2d():
    s = ora.Space((5, 4, 0), 2)
    assert s.m == (5, 4, 1) and s.n == (7, 6, 1) and s.shape == (1, 4, 5)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_split_step_against_dense_2d(p):
    ne = (5, 4)
    s = ora.Space(ne + (0,), p)
    Mx, Kx, _ = ref.restricted(ne[0], p)
    My, Ky, _ = ref.restricted(ne[1], p)
    tau = 0.09
    eta = tau * tau / 4
    K2 = np.kron(My, Kx) + np.kron(Ky, Mx)      # [y][x] row-major, x fastest
    G2 = np.kron(My + eta * Ky, Mx + eta * Kx)
    rng = np.random.default_rng(p)
    u, v = rng.standard_normal(s.shape), rng.standard_normal(s.shape)
    a = s.pwave_accel(u)
    np.testing.assert_allclose(a.ravel(), np.linalg.solve(np.kron(My, Mx), -K2 @ u.ravel()), rtol=1e-10, atol=1e-11)
    u1, v1, a1 = s.pwave_run(u, v, a, tau, 1)
    a_ref = np.linalg.solve(G2, -K2 @ (u + tau * v + eta * a).ravel())
    np.testing.assert_allclose(a1.ravel(), a_ref, rtol=1e-10, atol=1e-11)


def test_load_2d_against_scipy():
    ne, p, c, den = (6, 5), 2, (0.4, 0.55, 0.0), 0.03
    s = ora.Space(ne + (0,), p)
    g = s.load_gauss(1.7, c, den)
    gx = ref.load1d(ne[0], p, c[0], den)
    gy = ref.load1d(ne[1], p, c[1], den)
    np.testing.assert_allclose(g[0], 1.7 * np.outer(gy, gx), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("tau", [0.05, 2.0])
def test_sec3_eigenmode_recurrence_2d(tau):
    ne, p = (6, 5), 2
    s = ora.Space(ne + (0,), p)
    Mx, Kx, _ = ref.restricted(ne[0], p)
    My, Ky, _ = ref.restricted(ne[1], p)
    lx, Vx = sla.eigh(Kx, Mx)
    ly, Vy = sla.eigh(Ky, My)
    i, j = 2, 1
    mode = np.outer(Vy[:, j], Vx[:, i])[None]
    eta = tau * tau / 4
    k = lx[i] + ly[j]
    mt = (1 + eta * lx[i]) * (1 + eta * ly[j]) - eta * k   # the split mass on the mode
    u, v = mode.copy(), np.zeros_like(mode)
    a = s.pwave_accel(u)
    c_u, c_v, c_a = 1.0, 0.0, -k               # amplitude of u, v, a on the mode (consistent a0 = -k u0)
    for _ in range(12):
        u, v, a = s.pwave_run(u, v, a, tau, 1)
        ca_new = -k * (c_u + tau * c_v + eta * c_a) / (mt + eta * k)
        c_u, c_v, c_a = c_u + tau * c_v + eta * (c_a + ca_new), c_v + 0.5 * tau * (c_a + ca_new), ca_new
        # entries where the mode vanishes hold rounding noise of the field's size
        np.testing.assert_allclose(u, c_u * mode, rtol=1e-11, atol=1e-13 * abs(c_u) * np.abs(mode).max())
        np.testing.assert_allclose(a, c_a * mode, rtol=1e-10, atol=1e-12 * abs(c_a) * np.abs(mode).max())


@pytest.mark.parametrize("p,lam,mu", [(2, 1.0, 1.0), (3, 2.2, 0.6)])
def test_plane_strain_elasticity_against_2d_quadrature(p, lam, mu):
    ne = (4, 3)
    s = ora.Space(ne + (0,), p)
    S = ref.elastic_dense_2d(ne, p, lam, mu)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((3,) + s.shape)
    out = s.elastic_apply(lam, mu, U)
    N = s.shape[1] * s.shape[2]
    np.testing.assert_allclose(out[:2].ravel(), S @ U[:2].ravel(), rtol=1e-11, atol=1e-11)
    # u_z decouples: its block is mu times the 2D Laplacian form, and it does not feed u_x, u_y
    Mx, Kx, _ = ref.restricted(ne[0], p)
    My, Ky, _ = ref.restricted(ne[1], p)
    np.testing.assert_allclose(out[2].ravel(), mu * (np.kron(My, Kx) + np.kron(Ky, Mx)) @ U[2].ravel(),
                               rtol=1e-11, atol=1e-11)
    U2 = U.copy()
    U2[2] = 0
    np.testing.assert_allclose(s.elastic_apply(lam, mu, U2)[:2], out[:2], rtol=1e-12, atol=1e-12)
    assert N == np.prod(s.m)
