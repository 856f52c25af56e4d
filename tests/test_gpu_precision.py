"""The FP32 path with one FP64 residual correction per step: the residual
r = F - K p - G~ a is formed in FP64 from the FP32 state and the corrected
acceleration a + G~^{-1} r drives the update.  It must stay within the FP32
tolerances and bring the acceleration closer to the FP64 oracle than the
plain FP32 step does (the FP32 rounding of the RHS evaluation and of the
sweeps dominates the plain step's error; storage of the state does not)."""
import numpy as np
import pytest

from paper_1911_08158_gb300 import workloads as wl
from tests.cases import check_state, oracle_wave, rel_l2

pytestmark = pytest.mark.gpu


def _run(case, steps, **kw):
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, precision="fp32", **kw)
    sim.set_source(case.source)
    sim.set_gaussian_state(None, None)
    sim.step(steps)
    return sim, sim.get_state()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_residual_correction_improves_the_acceleration(p):
    case = wl.ricker_case(ne=(22, 19, 25), p=p, tau=2e-3, steps=0, seed=4, sigma=0.06)
    steps = 30
    ref = oracle_wave(case, steps)[steps]
    _, plain = _run(case, steps)
    _, corr = _run(case, steps, residual_correction=True)
    e_plain = [rel_l2(plain[k], ref[k]) for k in range(3)]
    e_corr = [rel_l2(corr[k], ref[k]) for k in range(3)]
    print("p=%d plain u,v,a %s  corrected %s" % (p, ["%.2e" % e for e in e_plain], ["%.2e" % e for e in e_corr]))
    base = 3e-5 if p == 4 else 1e-5
    check_state(corr, ref, "fp32", case.tau, base, "corrected p=%d" % p)
    # with the residual in FP64 the error left is the FP32 storage of the
    # state (~1e-7), for every degree and every field (measured 4-7e-8)
    assert max(e_corr) <= 1e-6
    assert e_corr[2] * 5 < e_plain[2]


def test_corrected_simulation_in_a_batch_equals_alone():
    from paper_1911_08158_gb300 import Simulation, batch_step
    case = wl.ricker_case(ne=(10, 12, 9), p=2, tau=3e-3, steps=0, seed=2, sigma=0.08)
    other = wl.pulse_case(ne=(8, 9, 10), p=2, tau=1e-2, steps=0)
    _, alone = _run(case, 20, residual_correction=True)
    a = Simulation(case.n_elem, case.p, case.tau, precision="fp32", residual_correction=True)
    a.set_source(case.source)
    a.set_gaussian_state(None, None)
    b = Simulation(other.n_elem, other.p, other.tau, precision="fp32")
    b.set_gaussian_state(other.u0, None)
    batch_step([a, b], 20)
    got = a.get_state()
    for k in range(3):
        assert np.array_equal(got[k], alone[k])
