"""Edge cases of the scalar-wave path against the oracle: the smallest
spaces (one unknown per axis), the largest line the kernels take (512
unknowns: 16 segments) along each axis, non-unit domain lengths, zero steps
and empty batches, and the size limit itself."""
import numpy as np
import pytest

import oracle as ora
from paper_1911_08158_gb300 import workloads as wl
from tests.cases import check_state, gpu_wave, oracle_wave

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((1, 1, 1), 2), ((2, 1, 3), 2), ((2, 3, 2), 1), ((1, 2, 1), 3)])
def test_smallest_spaces(ne, p, precision):
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=12, seed=1, sigma=0.2)
    ref = oracle_wave(case, 12)[12]
    _, got = gpu_wave(case, 12, precision)
    check_state(got[12], ref, precision, case.tau, TOL[precision] * (2 if precision == "fp64" else 3), "%s" % (ne,))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((510, 3, 2), 4), ((2, 512, 3), 2), ((3, 2, 510), 4)])
def test_longest_lines(ne, p, precision):
    """512 unknowns along one axis: 16 segments of 32 rows (K1 x or y sweep, K3 z sweep)."""
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=8, seed=2, sigma=0.05)
    assert max(n + p - 2 for n in ne) == 512
    ref = oracle_wave(case, 8)[8]
    _, got = gpu_wave(case, 8, precision)
    base = TOL[precision] * ((10 if precision == "fp64" else 3) if p == 4 else 1)
    check_state(got[8], ref, precision, case.tau, base, "%s p=%d" % (ne, p))


def test_lines_beyond_the_limit_are_rejected():
    from paper_1911_08158_gb300 import AdsError, Simulation
    with pytest.raises(AdsError) as e:
        Simulation((512, 4, 4), 3, 1e-3)           # 513 unknowns along x
    assert e.value.code == -5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_non_unit_domain(precision):
    from paper_1911_08158_gb300 import Simulation
    ne, p, L, tau, steps = (14, 11, 9), 3, (2.0, 0.7, 1.3), 3e-3, 20
    s = ora.Space(ne, p, L)
    u0 = s.project_gauss(1.0, (1.1, 0.3, 0.6), 0.05)
    v, a = s.zeros(), s.pwave_accel(u0)
    ref = s.pwave_run(u0, v, a, tau, steps)
    sim = Simulation(ne, p, tau, length=L, precision=precision)
    sim.set_gaussian_state(dict(amp=1.0, center=(1.1, 0.3, 0.6), den=0.05), None)
    sim.step(steps)
    check_state(sim.get_state(), tuple(s.pad(x) for x in ref), precision, tau,
                TOL[precision] * (2 if precision == "fp64" else 1), "L=%s" % (L,))


def test_zero_steps_and_empty_batch():
    from paper_1911_08158_gb300 import batch_step
    case = wl.pulse_case(ne=(6, 5, 4), p=2, steps=0)
    sim, got = gpu_wave(case, 0, "fp64")
    before = sim.get_state()
    sim.step(0)
    batch_step([sim], 0)
    batch_step([], 5)
    after = sim.get_state()
    assert sim.step_count == 0
    for x, y in zip(before, after):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_elasticity_long_lines(precision):
    """Long diagonal-block sweeps: 300 unknowns along x (FP32: 10 segments of
    32 rows; FP64: 7 segments of 44 rows in the 256-thread CTA).  The wide
    FP64 CTA (more than 8 segments) is covered by the 510- and 512-unknown
    lines of test_longest_lines and test_2d_long_lines_fp64."""
    from tests.cases import assert_parity, gpu_elastic, oracle_elastic
    case = wl.elastic_case(ne=(300, 4, 3), p=2, tau=4e-3, steps=6, seed=5, sigma=0.1)
    ref = oracle_elastic(case, 6)[6]
    _, got = gpu_elastic(case, 6, precision)
    assert_parity(got[6][0], ref[0], TOL[precision] * (2 if precision == "fp64" else 1), "U %s" % precision)


@pytest.mark.parametrize("boundary", ["dirichlet", "natural"])
def test_2d_long_lines_fp64(boundary):
    case = wl.ricker_case(ne=(3, 509, 0), p=3, tau=2e-3, steps=10, seed=3, sigma=0.05)
    ref = oracle_wave(case, 10, boundary=boundary)[10]
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, precision="fp64", boundary=boundary)
    sim.set_source(case.source)
    sim.set_gaussian_state(None, None)
    sim.step(10)
    check_state(sim.get_state(), ref, "fp64", case.tau, 2e-12, "2D %s" % boundary)


def test_batch_mixing_wide_and_narrow_fp64():
    """One batch of two FP64 simulations with different K1 instantiations
    (300 unknowns along x: 44-row segments; the small one: 32-row segments)."""
    from paper_1911_08158_gb300 import Simulation, batch_step
    cases = [wl.ricker_case(ne=(300, 3, 2), p=2, tau=2e-3, steps=0, seed=1, sigma=0.05),
             wl.ricker_case(ne=(10, 9, 8), p=2, tau=2e-3, steps=0, seed=2, sigma=0.05)]
    alone = [gpu_wave(c, 17, "fp64")[1][17] for c in cases]
    sims = []
    for c in cases:
        s = Simulation(c.n_elem, c.p, c.tau, precision="fp64")
        s.set_source(c.source)
        s.set_gaussian_state(None, None)
        sims.append(s)
    batch_step(sims, 17)
    for s, ref in zip(sims, alone):
        got = s.get_state()
        for k in range(3):
            assert np.array_equal(got[k], ref[k])
