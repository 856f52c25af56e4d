"""The natural (traction-free) boundary of Sec. 5 on the GPU, against the
oracle: every B-spline is an unknown (n_elem + p per axis)."""
import numpy as np
import pytest

import oracle as ora
from paper_1911_08158_gb300 import workloads as wl
from tests.cases import (assert_parity, check_state, derived_tols, gpu_elastic, gpu_wave, oracle_elastic, oracle_wave,
                         rel_l2)

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((10, 9, 8), 2), ((7, 9, 6), 3), ((33, 8, 10), 2)])
def test_elastic_natural_matches_oracle(ne, p, precision):
    case = wl.elastic_case(ne=ne, p=p, tau=4e-3, steps=10, seed=2, sigma=0.08)
    case.lam, case.mu, case.rho = 1.6, 0.8, 1.2
    src = dict(amp=2.0, center=(0.4, 0.55, 0.5), den=0.02, freq=8.0, t0=0.125, dir=(0.3, -0.5, 0.81))
    ref = oracle_elastic(case, 10, source=src, boundary="natural")[10]
    sim, got = gpu_elastic(case, 10, precision, source=src, boundary="natural")
    assert sim.shape == (3,) + tuple(n + p for n in ne[::-1])
    tol = TOL[precision]
    assert_parity(got[10][0], ref[0], tol, "%s U" % precision)
    tv, _ = derived_tols(ref[0], ref[1], ref[1], case.tau, tol)
    assert_parity(got[10][1], ref[1], tv, "%s V" % precision)


def test_uniform_velocity_translates_rigidly_on_gpu():
    from paper_1911_08158_gb300 import Simulation
    ne, p, tau = (9, 8, 10), 2, 0.02
    sim = Simulation(ne, p, tau, kind="elastic", lam=1.0, mu=1.0, rho=1.3, precision="fp64", boundary="natural")
    shape = sim.shape
    V0 = np.zeros(shape)
    V0[0], V0[2] = 0.7, -0.2
    sim.set_state(np.zeros(shape), V0)
    sim.step(30)
    U, V = sim.get_state()[:2]
    np.testing.assert_allclose(U, 30 * tau * V0, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(V, V0, rtol=1e-10, atol=1e-12)


def test_elastic_natural_invariant():
    case = wl.elastic_case(ne=(8, 9, 7), p=2, tau=5e-3, steps=0, seed=4, sigma=0.1)
    sim, got = gpu_elastic(case, 1, "fp64", boundary="natural")
    s = ora.Space(case.n_elem, case.p, natural=True)
    U, V = got[1]
    Eo = s.elastic_invariant(case.tau, case.lam, case.mu, case.rho, U, U - case.tau * V)
    k, pt, E = sim.energy()
    assert abs(E - Eo) <= 1e-11 * abs(Eo)
    for _ in range(3):
        sim.step(20)
        assert abs(sim.energy()[2] - E) <= 1e-11 * abs(E)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scalar_wave_natural_matches_oracle(precision):
    case = wl.ricker_case(ne=(14, 11, 12), p=3, tau=2e-3, steps=20, seed=6, sigma=0.06)
    ref = oracle_wave(case, 20, boundary="natural")[20]
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, precision=precision, boundary="natural")
    sim.set_source(case.source)
    sim.set_gaussian_state(None, None)
    sim.step(20)
    check_state(sim.get_state(), ref, precision, case.tau, TOL[precision] * (2 if precision == "fp64" else 1),
                "natural %s" % precision)


def test_operators_natural():
    import paper_1911_08158_gb300 as ads
    ne, p, tau = (7, 6, 5), 2, 0.03
    sim = ads.Simulation(ne, p, tau, boundary="natural")
    s = ora.Space(ne, p, natural=True)
    x = np.random.default_rng(2).standard_normal(s.shape)
    eta = tau * tau / 4
    for op, ref in ((ads.ADS_OP_MASS, s.apply_mass(x)), (ads.ADS_OP_STIFF, s.apply_lap(x)),
                    (ads.ADS_OP_MASS_SOLVE, s.solve_mass(x)),
                    (ads.ADS_OP_SPLIT_SOLVE, s.solve_kron((eta, eta, eta), x))):
        assert_parity(sim.apply(op, x), ref, 1e-12, "op %d" % op)
