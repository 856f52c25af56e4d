"""Pins of the oracle with the natural (traction-free) boundary of Sec. 5:
every B-spline kept, no Dirichlet restriction.

- Upsilon against brute-force 3D quadrature of 2 mu e(w):e(u) + lam div w div u
  on the full space (symmetric positive semidefinite, six-dimensional null space);
- the rigid-body modes (three translations, three infinitesimal rotations,
  represented exactly in the spline space through the Greville abscissae) are
  annihilated by Upsilon;
- a uniform initial velocity with no force moves the body rigidly: U^n = n tau V0;
- the discrete invariant of the alternating-triangular scheme is conserved;
- the scalar wave with natural boundary keeps a constant state constant and its
  split step matches a dense Kronecker solve.
"""
import numpy as np
import pytest

import oracle as ora
from tests import splines_ref as ref

NE = (3, 2, 3)


def greville(ne, p, L=1.0):
    t = ref.knots(ne, p, L)
    n = ne + p
    return np.array([t[a + 1:a + p + 1].mean() for a in range(n)])


def rigid_modes(s):
    """The six rigid-body displacement fields as coefficient arrays (3, nz, ny, nx)."""
    gx, gy, gz = (greville(s.ne[a], s.p, s.L[a]) for a in range(3))
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    one, zero = np.ones_like(X), np.zeros_like(X)
    modes = [np.stack([one, zero, zero]), np.stack([zero, one, zero]), np.stack([zero, zero, one]),
             np.stack([-Y, X, zero]), np.stack([zero, -Z, Y]), np.stack([Z, zero, -X])]
    return modes


@pytest.mark.parametrize("p,lam,mu", [(2, 1.0, 1.0), (3, 2.5, 0.7), (1, 0.4, 1.3)])
def test_upsilon_matches_direct_quadrature_natural(p, lam, mu):
    L = (1.0, 0.9, 1.3)
    s = ora.Space(NE, p, L, natural=True)
    assert s.m == tuple(n + p for n in NE)
    S = ref.elastic_dense(NE, p, lam, mu, L, natural=True)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((3,) + s.shape)
    np.testing.assert_allclose(s.elastic_apply(lam, mu, U).ravel(), S @ U.ravel(), rtol=1e-11, atol=1e-11)
    assert np.abs(S - S.T).max() < 1e-12
    ev = np.linalg.eigvalsh(S)
    scale = ev.max()
    assert np.sum(np.abs(ev) < 1e-10 * scale) == 6          # the rigid-body modes
    assert ev.min() > -1e-10 * scale                         # semidefinite


@pytest.mark.parametrize("p", [1, 2, 3])
def test_rigid_modes_are_annihilated(p):
    L = (1.0, 1.2, 0.8)
    s = ora.Space((4, 3, 3), p, L, natural=True)
    lam, mu = 1.7, 0.6
    for k, U in enumerate(rigid_modes(s)):
        out = s.elastic_apply(lam, mu, U)
        assert np.abs(out).max() < 1e-12 * (np.abs(U).max() + 1) * (lam + 2 * mu) * 10, "mode %d" % k
    # and a non-rigid linear field is not (sanity of the check itself)
    U = rigid_modes(s)[3]
    U[1] *= 2.0
    assert np.abs(s.elastic_apply(lam, mu, U)).max() > 1e-3


def test_uniform_velocity_translates_rigidly():
    s = ora.Space((4, 3, 5), 2, natural=True)
    lam, mu, rho, tau = 1.0, 1.0, 1.3, 0.02
    V0 = np.zeros((3,) + s.shape)
    V0[0], V0[2] = 0.7, -0.2
    U0 = np.zeros_like(V0)
    Up = s.elastic_start(tau, lam, mu, rho, U0, V0)
    U, Up = s.elastic_run(tau, lam, mu, rho, 25, U0, Up)
    np.testing.assert_allclose(U, 25 * tau * V0, rtol=1e-12, atol=1e-13)


def test_invariant_conserved_natural():
    s = ora.Space((4, 4, 3), 2, natural=True)
    lam, mu, rho, tau = 1.0, 0.8, 1.1, 0.05
    rng = np.random.default_rng(5)
    V0 = rng.standard_normal((3,) + s.shape) * 0.1
    U0 = rng.standard_normal((3,) + s.shape) * 0.01
    Up = s.elastic_start(tau, lam, mu, rho, U0, V0)
    U, Up = s.elastic_run(tau, lam, mu, rho, 1, U0, Up)
    E0 = s.elastic_invariant(tau, lam, mu, rho, U, Up)
    for _ in range(4):
        U, Up = s.elastic_run(tau, lam, mu, rho, 10, U, Up)
        E = s.elastic_invariant(tau, lam, mu, rho, U, Up)
        assert abs(E - E0) <= 1e-12 * abs(E0)


def test_scalar_wave_natural_constant_state_and_dense_step():
    s = ora.Space((3, 4, 2), 2, natural=True)
    u = np.ones(s.shape)
    v = np.zeros(s.shape)
    a = s.pwave_accel(u)
    assert np.abs(a).max() < 1e-12                         # K 1 = 0 without a boundary condition
    u2, v2, a2 = s.pwave_run(u, v, a, 0.1, 10)
    np.testing.assert_allclose(u2, u, rtol=0, atol=1e-12)
    # one split step against a dense Kronecker solve on the full space
    tau = 0.07
    eta = tau * tau / 4
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(s.shape), rng.standard_normal(s.shape)
    a = s.pwave_accel(u)
    Ms = [s.mat(ax, "M") for ax in range(3)]
    Ks = [s.mat(ax, "K") for ax in range(3)]
    K3 = ref.kron3(Ks[0], Ms[1], Ms[2]) + ref.kron3(Ms[0], Ks[1], Ms[2]) + ref.kron3(Ms[0], Ms[1], Ks[2])
    G = ref.kron3(*[Ms[ax] + eta * Ks[ax] for ax in range(3)])
    a1 = np.linalg.solve(G, -K3 @ (u + tau * v + eta * a).ravel())
    u1, v1, a1g = s.pwave_run(u, v, a, tau, 1)
    np.testing.assert_allclose(a1g.ravel(), a1, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(u1.ravel(), (u + tau * v + eta * (a + a1.reshape(s.shape))).ravel(), rtol=1e-11,
                               atol=1e-12)
