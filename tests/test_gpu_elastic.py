"""GPU parity of the linear-elasticity alternating-triangular step (Sec. 5,
eqs. decom/pre/corr/spill/gen) against the oracle, through the C ABI.

Displacement U^n: FP64 relative L2 <= 1e-12 per 10 steps (rounding grows
linearly with the step count), FP32 (state and sweeps in FP32, FP64 1D
factors) <= 1e-5.  The velocity (U^n - U^{n-1})/tau: the displacement bound
carried to the scheme's top frequency 2/tau (tests.cases.derived_tols)."""
import numpy as np
import pytest

import oracle as ora
from paper_1911_08158_gb300 import workloads as wl
from tests.cases import assert_parity, derived_tols, gpu_elastic, oracle_elastic, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _check(got, ref, precision, tau, n, what):
    base = TOL[precision] * (max(1.0, n / 10) if precision == "fp64" else 1.0)
    assert_parity(got[0], ref[0], base, what + " U")
    tv, _ = derived_tols(ref[0], ref[1], ref[1], tau, base)
    assert_parity(got[1], ref[1], tv, what + " V (tol %.1e)" % tv)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((12, 10, 9), 2), ((9, 11, 8), 3), ((7, 6, 9), 1)])
def test_velocity_pulse_matches_oracle(ne, p, precision):
    case = wl.elastic_case(ne=ne, p=p, tau=2e-3, steps=20, seed=2, sigma=0.1)
    ref = oracle_elastic(case, 20, checkpoints=(10,))
    _, got = gpu_elastic(case, 20, precision, checkpoints=(10,))
    for n in (10, 20):
        _check(got[n], ref[n], precision, case.tau, n, "%s step %d" % (precision, n))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_body_force_and_material(precision):
    case = wl.elastic_case(ne=(10, 12, 8), p=2, tau=3e-3, steps=15, seed=4, sigma=0.1)
    case.lam, case.mu, case.rho = 2.5, 0.7, 1.3
    case.v0 = None
    src = dict(amp=1.0, center=(0.45, 0.5, 0.55), den=2 * 0.08 ** 2, freq=8.0, t0=0.125, dir=(0.6, -0.3, 0.74))
    ref = oracle_elastic(case, 15, source=src)
    _, got = gpu_elastic(case, 15, precision, source=src)
    _check(got[15], ref[15], precision, case.tau, 15, precision)


def test_energies_and_invariant_conserved():
    case = wl.elastic_case(ne=(10, 9, 8), p=2, tau=0.02, steps=1, seed=5, sigma=0.12)
    sim, got = gpu_elastic(case, 1, "fp64")
    s = ora.Space(case.n_elem, case.p)
    U, V = (s.interior(x) for x in got[1])
    Up = U - case.tau * V
    k, pt, E = sim.energy()
    # kinetic / potential against the oracle's operators
    ko = 0.5 * case.rho * sum(float(np.sum(V[i] * s.apply_mass(V[i]))) for i in range(3))
    po = 0.5 * float(np.sum(U * s.elastic_apply(case.lam, case.mu, U)))
    Eo = s.elastic_invariant(case.tau, case.lam, case.mu, case.rho, U, Up)
    assert abs(k - ko) <= 1e-11 * ko and abs(pt - po) <= 1e-11 * po and abs(E - Eo) <= 1e-11 * Eo
    for _ in range(4):
        sim.step(25)
        assert abs(sim.energy()[2] - E) <= 1e-10 * E


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_elastic_checkpoint_bitwise(precision):
    case = wl.elastic_case(ne=(8, 9, 10), p=2, tau=2e-3, steps=10, seed=6, sigma=0.1)
    simA, gotA = gpu_elastic(case, 10, precision)
    simB, _ = gpu_elastic(case, 4, precision)
    blob = simB.checkpoint()
    simC, _ = gpu_elastic(case, 0, precision)
    simC.restore(blob)
    simC.step(6)
    for x, y in zip(simC.get_state()[:2], gotA[10]):
        assert np.array_equal(x, y)


def test_96cubed_elasticity_100_steps():
    """The elasticity configuration at its full size and length (96^3
    elements, p = 2, three components, tau = 2e-3, 100 steps, seeded vector
    Gaussian velocity pulse), FP64 and FP32 against the oracle after 10 and
    after 100 steps."""
    case = wl.elastic_case(ne=96, p=2, tau=2e-3, steps=100)
    ref = oracle_elastic(case, 100, checkpoints=(10,))
    for precision in ("fp64", "fp32"):
        _, got = gpu_elastic(case, 100, precision, checkpoints=(10,))
        for n in (10, 100):
            _check(got[n], ref[n], precision, case.tau, n, "%s step %d" % (precision, n))
            print("96^3 elasticity %s rel-L2 U at %d: %.3e" % (precision, n, rel_l2(got[n][0], ref[n][0])))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne", [(65, 14, 9), (129, 129, 4)])
def test_segment_lengths(ne, precision):
    """Grids whose lines take 33-row segments (65 unknowns along x) and, in
    FP32, 44-row segments (129 x 129 planes, which the elastic K1 also splits
    into row tiles because three such planes exceed shared memory) in the
    fused elastic step, against the oracle."""
    case = wl.elastic_case(ne=ne, p=2, tau=3e-3, steps=6, seed=7, sigma=0.1)
    ref = oracle_elastic(case, 6)[6]
    _, got = gpu_elastic(case, 6, precision)
    _check(got[6], ref, precision, case.tau, 6, "%s %s" % (precision, ne))
