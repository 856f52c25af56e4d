"""2D problems (n_elem[2] = 0) on the GPU against the oracle: the same
kernels run with one constant function along z."""
import numpy as np
import pytest

from paper_1911_08158_gb300 import workloads as wl
from tests.cases import assert_parity, check_state, derived_tols, gpu_elastic, gpu_wave, oracle_elastic, oracle_wave

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((32, 32, 0), 2), ((45, 29, 0), 3), ((128, 97, 0), 2)])
def test_2d_ricker_matches_oracle(ne, p, precision):
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=30, seed=5, sigma=0.05)
    ref = oracle_wave(case, 30)[30]
    sim, got = gpu_wave(case, 30, precision)
    assert sim.shape == (1, ne[1] + p, ne[0] + p)
    check_state(got[30], ref, precision, case.tau, TOL[precision] * (3 if precision == "fp64" else 1),
                "2D %s %s" % (ne, precision))


@pytest.mark.parametrize("boundary", ["dirichlet", "natural"])
def test_2d_pulse(boundary):
    case = wl.pulse_case(ne=(24, 20, 0), p=2, tau=1e-2, steps=20)
    ref = oracle_wave(case, 20, boundary=boundary)[20]
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, precision="fp64", boundary=boundary)
    sim.set_gaussian_state(case.u0, None)
    sim.step(20)
    check_state(sim.get_state(), ref, "fp64", case.tau, 3e-12, "2D pulse %s" % boundary)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2d_elasticity(precision):
    case = wl.elastic_case(ne=(20, 17, 0), p=2, tau=4e-3, steps=15, seed=3, sigma=0.08)
    ref = oracle_elastic(case, 15)[15]
    _, got = gpu_elastic(case, 15, precision)
    tol = TOL[precision]
    assert_parity(got[15][0], ref[0], tol, "%s U" % precision)
    tv, _ = derived_tols(ref[0], ref[1], ref[1], case.tau, tol)
    assert_parity(got[15][1], ref[1], tv, "%s V" % precision)


def test_2d_in_a_batch_equals_alone():
    from paper_1911_08158_gb300 import batch_step
    a2 = wl.ricker_case(ne=(40, 33, 0), p=2, tau=2e-3, steps=0, seed=1, sigma=0.05)
    b3 = wl.ricker_case(ne=(12, 10, 9), p=2, tau=2e-3, steps=0, seed=2, sigma=0.05)
    sims, alone = [], []
    for c in (a2, b3):
        _, got = gpu_wave(c, 19, "fp32")
        alone.append(got[19])
    from paper_1911_08158_gb300 import Simulation
    for c in (a2, b3):
        s = Simulation(c.n_elem, c.p, c.tau, precision="fp32")
        s.set_source(c.source)
        s.set_gaussian_state(None, None)
        sims.append(s)
    batch_step(sims, 19)
    for s, ref in zip(sims, alone):
        got = s.get_state()
        for k in range(3):
            assert np.array_equal(got[k], ref[k])
