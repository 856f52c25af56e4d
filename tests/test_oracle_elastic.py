"""Pins of the oracle's linear-elasticity path (Sec. 5-6).

Upsilon is checked against a brute-force 3D quadrature of the bilinear form
2 mu e(w):e(u) + lam div w div u (independent of the Kronecker block
formulas); the alternating-triangular step against a dense block-triangular
solve built on that brute-force matrix; the scheme against its exactly
conserved discrete invariant (a priori estimate of Sec. 5.1, eq. equality), the stability
condition D - tau^2 Ups / 4 > 0, boundedness for large tau and second order."""
import numpy as np
import pytest

import oracle as ora
from tests import splines_ref as ref

NE = (3, 3, 2)


@pytest.mark.parametrize("p,lam,mu", [(2, 1.0, 1.0), (2, 2.5, 0.7), (3, 0.3, 1.9), (1, 1.0, 1.0)])
def test_upsilon_matches_direct_quadrature(p, lam, mu):
    L = (1.0, 1.2, 0.8)
    s = ora.Space(NE, p, L)
    S = ref.elastic_dense(NE, p, lam, mu, L)
    N = np.prod(s.m)
    rng = np.random.default_rng(7)
    U = rng.standard_normal((3,) + s.shape)
    np.testing.assert_allclose(s.elastic_apply(lam, mu, U).ravel(), S @ U.ravel(), rtol=1e-11, atol=1e-11)
    assert np.abs(S - S.T).max() < 1e-12
    assert np.linalg.eigvalsh(S).min() > 0       # SPD with Dirichlet
    # single blocks agree with the slices of the dense matrix
    for i in range(3):
        for j in range(3):
            Uj = U[j]
            out = s.elastic_block(lam, mu, i, j, Uj)
            np.testing.assert_allclose(out.ravel(), S[i * N:(i + 1) * N, j * N:(j + 1) * N] @ Uj.ravel(),
                                       rtol=1e-11, atol=1e-11)


def _dense_atm(s, S, tau, lam, mu, rho):
    """D = (rho M + tau^2/2 Ups1~)(rho M)^{-1}(rho M + tau^2/2 Ups2~) with the
    diagonal blocks factored as eq. (spill)."""
    N = np.prod(s.m)
    Ms = [s.mat(a, "M") for a in range(3)]
    Ks = [s.mat(a, "K") for a in range(3)]
    M3 = ref.kron3(*Ms)
    Z = np.zeros((N, N))

    def Lt(i):
        f = [Ms[a] + tau ** 2 * ((2 * mu + lam) if a == i else mu) / (4 * rho) * Ks[a] for a in range(3)]
        return rho * ref.kron3(*f)

    blk = lambda i, j: S[i * N:(i + 1) * N, j * N:(j + 1) * N]
    Lo = np.block([[Lt(i) if i == j else (tau ** 2 / 2 * blk(i, j) if i > j else Z) for j in range(3)]
                   for i in range(3)])
    Up = np.block([[Lt(i) if i == j else (tau ** 2 / 2 * blk(i, j) if i < j else Z) for j in range(3)]
                   for i in range(3)])
    RM = np.kron(np.eye(3), rho * M3)
    return Lo, Up, RM


@pytest.mark.parametrize("tau", [0.05, 3.0])
def test_atm_step_matches_dense_block_triangular(tau):
    p, lam, mu, rho = 2, 1.0, 1.0, 1.3
    s = ora.Space(NE, p)
    S = ref.elastic_dense(NE, p, lam, mu)
    Lo, Up, RM = _dense_atm(s, S, tau, lam, mu, rho)
    assert np.abs(Up - Lo.T).max() < 1e-12
    rng = np.random.default_rng(3)
    Uc = rng.standard_normal((3,) + s.shape)
    Upv = rng.standard_normal((3,) + s.shape)
    U1, U0 = s.elastic_run(tau, lam, mu, rho, 1, Uc, Upv)
    D = Lo @ np.linalg.solve(RM, Up)
    delta = np.linalg.solve(D, -tau ** 2 * (S @ Uc.ravel()))
    np.testing.assert_allclose(U1.ravel(), 2 * Uc.ravel() - Upv.ravel() + delta, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(U0, Uc, atol=0)
    # stability condition of the a priori estimate (sigma >= 1/4 form)
    Dm = D - tau ** 2 / 4 * S
    assert np.linalg.eigvalsh(0.5 * (Dm + Dm.T)).min() > 0


def _pulse(s, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    c = rng.uniform(0.3, 0.7, 3)
    g = s.project_gauss(1.0, c, 2 * 0.15 ** 2)
    return np.stack([a[i] * g for i in range(3)])


@pytest.mark.parametrize("tau", [0.02, 1.0, 50.0])
def test_atm_invariant_conserved_and_bounded(tau):
    p, lam, mu, rho = 2, 1.0, 1.0, 1.0
    s = ora.Space((5, 4, 4), p)
    V0 = _pulse(s)
    U0 = np.zeros_like(V0)
    Up = s.elastic_start(tau, lam, mu, rho, U0, V0)
    np.testing.assert_allclose(Up, -tau * V0, atol=0)      # U0 = 0: U^-1 = -tau V0
    Uc, Upv = U0, Up
    U1, _ = s.elastic_run(tau, lam, mu, rho, 1, Uc, Upv)
    E0 = s.elastic_invariant(tau, lam, mu, rho, U1, Uc)
    Uc, Upv = U1, Uc
    for _ in range(8):
        Un, Upn = s.elastic_run(tau, lam, mu, rho, 25, Uc, Upv)
        E = s.elastic_invariant(tau, lam, mu, rho, Un, Upn)
        # invariant at level n+1/2 uses (U^{n+1}, U^n) = (Un, Upn)
        assert abs(E - E0) <= 1e-10 * E0, (E, E0)
        Uc, Upv = Un, Upn


def test_atm_second_order_in_time():
    p, lam, mu, rho, T = 2, 1.0, 1.0, 1.0, 0.3
    s = ora.Space((6, 5, 5), p)
    V0 = _pulse(s, 1)
    U0 = np.zeros_like(V0)

    def run(N):
        tau = T / N
        Up = s.elastic_start(tau, lam, mu, rho, U0, V0)
        U, _ = s.elastic_run(tau, lam, mu, rho, N, U0, Up)
        return U

    ref_u = run(640)
    errs = [np.linalg.norm(run(N) - ref_u) for N in (20, 40, 80)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), rates


def test_atm_body_force_enters_at_level_n():
    """eq. gen: D (U^{n+1} - 2U^n + U^{n-1}) / tau^2 + Ups U^n = f^n, with
    f^n = r(t_n) dir g; from a zero state one step gives D delta = tau^2 f^n."""
    p, lam, mu, rho, tau = 2, 1.3, 0.8, 1.1, 0.04
    s = ora.Space(NE, p)
    S = ref.elastic_dense(NE, p, lam, mu)
    Lo, Up, RM = _dense_atm(s, S, tau, lam, mu, rho)
    D = Lo @ np.linalg.solve(RM, Up)
    G = s.load_gauss(1.0, (0.4, 0.5, 0.6), 0.05)
    d = np.array([0.3, -0.5, 0.8])
    z = s.zeros(3)
    U1, _ = s.elastic_run(tau, lam, mu, rho, 1, z, z, G=G, direction=d, rick=(8.0, 0.125), step0=5)
    f = ora.ricker(8.0, 0.125, 5 * tau) * np.concatenate([d[i] * G.ravel() for i in range(3)])
    np.testing.assert_allclose(U1.ravel(), np.linalg.solve(D, tau ** 2 * f), rtol=1e-9, atol=1e-14)
    # start-up with a force: U^{-1} = U0 - tau V0 + tau^2/2 (rho M)^{-1} f(t0)
    Um = s.elastic_start(tau, lam, mu, rho, z, z, G=G, direction=d, rick=(8.0, 0.125), t0=0.0)
    M3 = np.kron(np.eye(3), rho * ref.kron3(*[s.mat(a, "M") for a in range(3)]))
    f0 = ora.ricker(8.0, 0.125, 0.0) * np.concatenate([d[i] * G.ravel() for i in range(3)])
    np.testing.assert_allclose(Um.ravel(), 0.5 * tau ** 2 * np.linalg.solve(M3, f0), rtol=1e-9, atol=1e-16)
