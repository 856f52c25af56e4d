"""Pins of the oracle's 3D scalar P-wave path (Sec. 2-4, Appendix).

Brute force: the oracle's Kronecker operators and directional solves against
dense matrices assembled from SciPy-evaluated 1D matrices.  Time scheme:
exact conservation of the discrete invariant (Newmark with the split mass),
the Sec. 3 eigenmode reduction, boundedness for huge tau, and second order in
time against the exact semi-discrete solution."""
import numpy as np
import pytest

import oracle as ora
from tests import splines_ref as ref

NE = (5, 4, 3)


def _dense(ne, p, L=(1.0, 1.0, 1.0)):
    Ms, Ks = [], []
    for a in range(3):
        M, K, _ = ref.restricted(ne[a], p, L[a])
        Ms.append(M); Ks.append(K)
    return Ms, Ks


@pytest.mark.parametrize("p", [1, 2, 3])
def test_operators_match_dense_kronecker(p):
    L = (1.0, 0.7, 1.3)
    s = ora.Space(NE, p, L)
    Ms, Ks = _dense(NE, p, L)
    M3 = ref.kron3(*Ms)
    K3 = ref.kron3(Ks[0], Ms[1], Ms[2]) + ref.kron3(Ms[0], Ks[1], Ms[2]) + ref.kron3(Ms[0], Ms[1], Ks[2])
    rng = np.random.default_rng(p)
    u = rng.standard_normal(s.shape)
    np.testing.assert_allclose(s.apply_mass(u).ravel(), M3 @ u.ravel(), atol=1e-14)
    np.testing.assert_allclose(s.apply_lap(u, 2.5).ravel(), 2.5 * K3 @ u.ravel(), atol=1e-11)
    d = (0.3, 0.01, 0.07)
    G = ref.kron3(*[Ms[a] + d[a] * Ks[a] for a in range(3)])
    np.testing.assert_allclose(s.solve_kron(d, u).ravel(), np.linalg.solve(G, u.ravel()), rtol=1e-9,
                               atol=1e-9)
    np.testing.assert_allclose(s.solve_mass(u).ravel(), np.linalg.solve(M3, u.ravel()), rtol=1e-9,
                               atol=1e-9)


def test_load_is_separable_and_projection_factorises():
    # a separable Gaussian: the 3D tensor Gauss rule factorises into 1D rules
    p, ne, c, den = 2, (6, 5, 7), (0.4, 0.55, 0.6), 0.02
    s = ora.Space(ne, p)
    F = s.load_gauss(1.7, c, den)
    g = [ref.load1d(ne[a], p, c[a], den) for a in range(3)]
    F1 = 1.7 * np.einsum("k,j,i->kji", g[2], g[1], g[0])
    np.testing.assert_allclose(F, F1, rtol=1e-12, atol=1e-17)
    # projection = (Mx^-1 gx) (x) (My^-1 gy) (x) (Mz^-1 gz)
    P = s.project_gauss(1.0, c, den)
    Ms, _ = _dense(ne, p)
    pr = [np.linalg.solve(Ms[a], g[a]) for a in range(3)]
    np.testing.assert_allclose(P, np.einsum("k,j,i->kji", pr[2], pr[1], pr[0]), rtol=1e-10, atol=1e-14)


def test_projection_reproduces_the_spline_space():
    # L2 projection of a function already in the space is the identity: take
    # the projection of a Gaussian, re-project its own load -> same coefficients
    s = ora.Space((6, 6, 6), 3)
    P = s.project_gauss(1.0, (0.5, 0.5, 0.5), 0.01)
    np.testing.assert_allclose(s.solve_mass(s.apply_mass(P)), P, atol=1e-12)


def test_first_step_uses_source_at_t_n_plus_1():
    p, tau = 2, 0.01
    s = ora.Space(NE, p)
    Ms, Ks = _dense(NE, p)
    G = s.load_gauss(1.0, (0.5, 0.45, 0.5), 2 * 0.1 ** 2)
    z = s.zeros()
    u, v, a = s.pwave_run(z, z, z, tau, 1, step0=3, G=G, rick=(8.0, 0.125))
    eta = tau * tau / 4
    Gt = ref.kron3(*[Ms[i] + eta * Ks[i] for i in range(3)])
    a1 = np.linalg.solve(Gt, ora.ricker(8.0, 0.125, 4 * tau) * G.ravel())
    np.testing.assert_allclose(a.ravel(), a1, rtol=1e-10, atol=1e-16)
    np.testing.assert_allclose(u.ravel(), eta * a1, rtol=1e-10, atol=1e-20)
    np.testing.assert_allclose(v.ravel(), 0.5 * tau * a1, rtol=1e-10, atol=1e-20)


def _mode(ne, p, k=(0, 0, 0)):
    import scipy.linalg as sl
    Ms, Ks = _dense(ne, p)
    lam, vec = [], []
    for a in range(3):
        w, V = sl.eigh(Ks[a], Ms[a])
        lam.append(w[k[a]]); vec.append(V[:, k[a]])
    U0 = np.einsum("k,j,i->kji", vec[2], vec[1], vec[0])
    return U0, lam


def test_eigenmode_stays_a_mode_and_follows_scalar_newmark():
    """Sec. 3: with K_xi v = lam_xi M_xi v the split operator is diagonal,
    G~ -> prod(1 + eta lam_xi) M and K -> sum(lam_xi) M."""
    p, tau, ne = 3, 0.05, (6, 5, 4)
    U0, lam = _mode(ne, p, (1, 0, 2))
    s = ora.Space(ne, p)
    eta = tau * tau / 4
    gm, k = np.prod([1 + eta * l for l in lam]), np.sum(lam)
    al, ald, ala = 1.0, 0.0, -k
    u, v = U0.copy(), np.zeros_like(U0)
    a = s.pwave_accel(u)
    np.testing.assert_allclose(a, -k * U0, rtol=1e-9, atol=1e-9)
    for n in range(30):
        u, v, a = s.pwave_run(u, v, a, tau, 1, step0=n)
        an = -k * (al + tau * ald + eta * ala) / gm
        al, ald, ala = al + tau * ald + eta * (ala + an), ald + 0.5 * tau * (ala + an), an
        np.testing.assert_allclose(u, al * U0, atol=1e-12 * np.abs(U0).max())
        np.testing.assert_allclose(v, ald * U0, atol=1e-11 * np.abs(U0).max() * np.sqrt(k))


@pytest.mark.parametrize("tau", [0.01, 1.0, 10.0, 100.0])
def test_discrete_invariant_is_conserved_and_bounded(tau):
    """f = 0: after the first step the split scheme is Newmark on (G~ - eta K, K),
    whose energy 1/2 v^T (G~ - eta K) v + 1/2 u^T K u is exactly conserved; this
    is the unconditional stability of Sec. 3 (also for huge tau, Sec. 3 limits)."""
    p = 2
    s = ora.Space((6, 5, 4), p)
    u = s.project_gauss(1.0, (0.45, 0.5, 0.55), 0.01)
    v = np.zeros_like(u)
    a = s.pwave_accel(u)
    nsteps = 1000 if tau >= 1.0 else 200
    u, v, a = s.pwave_run(u, v, a, tau, 1)
    k, pt, km = s.pwave_energy(u, v, tau)
    E1 = km + pt
    for chunk in range(10):
        u, v, a = s.pwave_run(u, v, a, tau, nsteps // 10, step0=1 + chunk * nsteps // 10)
        k, pt, km = s.pwave_energy(u, v, tau)
        assert abs(km + pt - E1) <= 1e-11 * E1
        # bounded: both parts of the invariant are nonnegative and below E1
        assert -1e-12 * E1 <= pt <= E1 * (1 + 1e-11) and -1e-12 * E1 <= km <= E1 * (1 + 1e-11)


def test_second_order_in_time_against_semi_discrete_exact():
    """Lowest 3D eigenmode: the semi-discrete solution is cos(sqrt(k) t) U0,
    so the full error is the time error alone; it must fall 4x per halving."""
    p, ne, T = 3, (6, 6, 6), 0.9
    U0, lam = _mode(ne, p)
    k = np.sum(lam)
    s = ora.Space(ne, p)
    errs = []
    for N in (20, 40, 80, 160):
        tau = T / N
        u, v = U0.copy(), np.zeros_like(U0)
        a = s.pwave_accel(u)
        u, v, a = s.pwave_run(u, v, a, tau, N)
        errs.append(np.abs(u - np.cos(np.sqrt(k) * T) * U0).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), rates


def test_second_order_in_time_general_data():
    """Gaussian initial data (many modes) against a fine-tau run."""
    p, ne, T = 2, (8, 7, 6), 0.4
    s = ora.Space(ne, p)
    u0 = s.project_gauss(1.0, (0.5, 0.5, 0.5), 0.01)
    a0 = s.pwave_accel(u0)
    z = np.zeros_like(u0)
    ref_u, _, _ = s.pwave_run(u0, z, a0, T / 640, 640)
    errs = []
    for N in (20, 40, 80):
        u, _, _ = s.pwave_run(u0, z, a0, T / N, N)
        errs.append(np.linalg.norm(u - ref_u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), rates


def _interior_basis_at_gauss(ne, p, q):
    """Gauss points and weights on [0, 1] (q per element) and the values of the
    Dirichlet-restricted basis there (rows: points, columns: interior functions)."""
    gx, gw = np.polynomial.legendre.leggauss(q)
    X, Wq, B = [], [], []
    for e in range(ne):
        a, h = e / ne, 1.0 / ne
        for xg, wg in zip(gx, gw):
            x = a + 0.5 * h * (xg + 1)
            N, _ = ora.basis(ne, p, p + e, x)
            X.append(x)
            Wq.append(0.5 * h * wg)
            B.append(N[1:-1])
    return np.array(X), np.array(Wq), np.array(B)


@pytest.mark.parametrize("p,nes,T,N", [(1, (6, 12, 24), 0.3, 1600), (2, (6, 12, 24), 0.3, 1600),
                                       (3, (4, 8, 16), 0.1, 4000)])
def test_standing_wave_converges_in_space_at_order_p_plus_1(p, nes, T, N):
    """Spatial order of the whole scheme (soft pin; the paper states no rate):
    u = sin(pi x) sin(pi y) sin(pi z) cos(sqrt(3) pi t) solves u_tt = Laplace u
    with homogeneous Dirichlet data.  L2-project u(0), step with a time step
    small enough that the O(tau^2) error stays well below the spatial one, and
    measure the L2 error at T by tensor Gauss quadrature: it falls as h^(p+1)
    (measured log2 ratios: p=1 2.00 2.00, p=2 3.40 3.15, p=3 4.24 4.09)."""
    errs = []
    for ne in nes:
        s = ora.Space((ne, ne, ne), p)
        X, Wq, B = _interior_basis_at_gauss(ne, p, p + 3)
        f = np.sin(np.pi * X)
        c = np.linalg.solve(s.mat(0, "M"), B.T @ (Wq * f))       # 1D projection of sin(pi x)
        U0 = np.einsum("k,j,i->kji", c, c, c)                       # the 3D projection is its product
        u, _, _ = s.pwave_run(U0, np.zeros_like(U0), s.pwave_accel(U0), T / N, N)
        uh = np.einsum("kbc,ak->abc", np.einsum("kjc,bj->kbc", u @ B.T, B), B)
        exact = np.einsum("a,b,c->abc", f, f, f) * np.cos(np.sqrt(3) * np.pi * T)
        w3 = np.einsum("a,b,c->abc", Wq, Wq, Wq)
        errs.append(np.sqrt(np.sum(w3 * (uh - exact) ** 2)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - (p + 1)) < 0.2, (errs, rates)
    assert all(p + 1 - 0.2 < r < p + 1 + 0.5 for r in rates), (errs, rates)


def test_thread_count_does_not_change_results():
    """The oracle's OpenMP loops run over independent lines: 1 thread and all
    threads give bitwise equal steps (the benchmark times both)."""
    from paper_1911_08158_gb300 import workloads as wl
    case = wl.ricker_case(ne=(14, 12, 10), p=3, tau=2e-3, steps=3, seed=3, sigma=0.08)
    s = ora.Space(case.n_elem, case.p)
    G = s.load_gauss(case.source["amp"], case.source["center"], case.source["den"])
    z = s.zeros()
    a = s.pwave_accel(z, 0.0, 1.0, G)
    allc = ora.num_threads()
    try:
        ora.set_num_threads(1)
        one = s.pwave_run(z, z, a, case.tau, 3, step0=0, G=G)
    finally:
        ora.set_num_threads(allc)
    many = s.pwave_run(z, z, a, case.tau, 3, step0=0, G=G)
    for x, y in zip(one, many):
        assert np.array_equal(x, y)
