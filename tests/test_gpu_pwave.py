"""GPU parity of the scalar P-wave path against the oracle, through the C ABI.

Tolerances (relative L2 over the field, and every element within 10x the
tolerance of the field's maximum):
  - FP64 path: 1e-12 on u, v (p <= 3).  For p = 4 the solution moves by
    ~2e-12 under ulp-level differences of the 1D matrices (two independent
    FP64 evaluations of M, K that both match the exact rational stencils to a
    few ulps), so p = 4 uses 1e-11.  Long runs: 1e-12 per 10 steps
    (rounding accumulates linearly in the step count).
  - FP32 path (FP32 state and sweeps, FP64 1D factors rounded): 1e-5 on the
    displacement u for p <= 3.  FP32 rounding errors of the directional
    solves scale with cond(M_xi), which grows ~2.8x per degree (p = 3: 21,
    p = 4: 58), so p = 4 uses 3e-5.
  - velocity v and acceleration a: the displacement tolerance carried to the
    scheme's highest frequency 2/tau (tests.cases.derived_tols)."""
import os

import numpy as np
import pytest

import oracle as ora
from paper_1911_08158_gb300 import workloads as wl
from tests.cases import assert_parity, check_state, gpu_wave, oracle_wave, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _sim(ne, p, tau=0.01, precision="fp64", **kw):
    from paper_1911_08158_gb300 import Simulation
    return Simulation(ne, p, tau, precision=precision, **kw)


@pytest.mark.parametrize("ne,p", [((5, 4, 3), 1), ((5, 4, 3), 2), ((6, 5, 4), 3), ((7, 6, 5), 4),
                                  ((33, 17, 9), 2), ((40, 31, 27), 3), ((1, 2, 3), 2)])
def test_operators_match_oracle(ne, p):
    import paper_1911_08158_gb300 as ads
    tau = 0.03
    sim = _sim(ne, p, tau)
    s = ora.Space(ne, p)
    rng = np.random.default_rng(sum(ne) + p)
    x = rng.standard_normal(s.shape)
    xf = s.pad(x)
    eta = tau * tau / 4
    for op, ref in ((ads.ADS_OP_MASS, s.apply_mass(x)), (ads.ADS_OP_STIFF, s.apply_lap(x)),
                    (ads.ADS_OP_MASS_SOLVE, s.solve_mass(x)),
                    (ads.ADS_OP_SPLIT_SOLVE, s.solve_kron((eta, eta, eta), x))):
        got = sim.apply(op, xf)
        assert_parity(got, s.pad(ref), 1e-12, "op %d" % op)
        # boundary coefficients stay zero
        assert np.all(got[0] == 0) and np.all(got[:, 0] == 0) and np.all(got[..., -1] == 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pulse_16cubed_matches_oracle(precision):
    """16^3 elements, p = 2, tau = 1e-2, Gaussian pulse, 20 steps."""
    case = wl.pulse_case()
    ref = oracle_wave(case, 20, checkpoints=(10,))
    _, got = gpu_wave(case, 20, precision, checkpoints=(10,))
    for n in (10, 20):
        tol = TOL[precision] * (n / 10 if precision == "fp64" else 1)
        check_state(got[n], ref[n], precision, case.tau, tol, "%s step %d" % (precision, n))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((24, 20, 18), 3), ((37, 29, 11), 2), ((9, 40, 13), 1), ((14, 12, 10), 4)])
def test_ricker_source_ragged_grids(ne, p, precision):
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=40, seed=3, sigma=0.05)
    ref = oracle_wave(case, 40, checkpoints=(10,))
    _, got = gpu_wave(case, 40, precision, checkpoints=(10,))
    base = TOL[precision] * ((10 if precision == "fp64" else 3) if p == 4 else 1)
    for n in (10, 40):
        tol = base * (n / 10 if precision == "fp64" else 1)
        check_state(got[n], ref[n], precision, case.tau, tol, "%s step %d" % (precision, n))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((32, 31, 30), 3), ((64, 20, 16), 3), ((33, 65, 20), 2), ((97, 130, 4), 2)])
def test_33_row_segments(ne, p, precision):
    """Axes with 32 s + 1 unknowns (33, 65, 97 ...) run the line solves with
    33-row segments (one segment fewer per line); single-segment lines, ragged
    tails on the other axes and (97 x 130 planes in FP64) the row-tiled K1
    with the separate y sweep are covered."""
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=20, seed=8, sigma=0.05)
    ref = oracle_wave(case, 20)
    _, got = gpu_wave(case, 20, precision)
    check_state(got[20], ref[20], precision, case.tau, TOL[precision] * (2 if precision == "fp64" else 1),
                "%s %s p=%d" % (precision, ne, p))


@pytest.mark.parametrize("tile", [None, "16"])
@pytest.mark.parametrize("ne,p", [((128, 129, 4), 3), ((130, 129, 3), 2)])
def test_44_row_segments(ne, p, tile, monkeypatch):
    """FP32 planes of 129..132 unknowns per axis take 44-row segments (3 per
    line, so that every line group of K1 runs in one round), the FP64 set-up
    sweeps of the same simulation too; the whole-plane K1 and the row-tiled
    K1 with the separate y sweep (K2) are covered."""
    if tile:
        monkeypatch.setenv("ADS_RHS_TILE", tile)
    else:
        monkeypatch.delenv("ADS_RHS_TILE", raising=False)
    case = wl.ricker_case(ne=ne, p=p, tau=2e-3, steps=8, seed=11, sigma=0.05)
    ref = oracle_wave(case, 8)
    _, got = gpu_wave(case, 8, "fp32")
    check_state(got[8], ref[8], "fp32", case.tau, TOL["fp32"], "%s p=%d tile %s" % (ne, p, tile))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_and_tiled_rhs_agree(precision, monkeypatch):
    """The fused K1 (tile = whole y extent, y sweep inside) and the tiled K1 +
    separate y sweep compute the same step."""
    case = wl.ricker_case(ne=(20, 30, 12), p=2, tau=2e-3, steps=12, seed=5, sigma=0.05)
    ref = oracle_wave(case, 12)
    outs = []
    for tile in (None, "4,3", "7,2"):
        if tile:
            monkeypatch.setenv("ADS_RHS_TILE", tile)
        else:
            monkeypatch.delenv("ADS_RHS_TILE", raising=False)
        _, got = gpu_wave(case, 12, precision)
        outs.append(got[12])
        check_state(got[12], ref[12], precision, case.tau, TOL[precision] * (2 if precision == "fp64" else 1),
                    "tile %s" % tile)


def test_energy_invariant_conserved_on_gpu():
    case = wl.pulse_case(ne=(12, 10, 9), p=3, tau=0.05)
    sim, _ = gpu_wave(case, 1, "fp64")
    k, pt, km = sim.energy()
    E1 = km + pt
    s = ora.Space(case.n_elem, case.p)
    u, v, a = sim.get_state()
    ko, po, kmo = s.pwave_energy(s.interior(u), s.interior(v), case.tau)
    assert abs(k - ko) <= 1e-12 * abs(ko) and abs(pt - po) <= 1e-12 * abs(po) and abs(km - kmo) <= 1e-12 * abs(kmo)
    for _ in range(5):
        sim.step(40)
        k, pt, km = sim.energy()
        assert abs(km + pt - E1) <= 1e-11 * E1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_bitwise(precision):
    case = wl.ricker_case(ne=(18, 16, 14), p=2, tau=2e-3, steps=10, seed=1, sigma=0.05)
    simA, gotA = gpu_wave(case, 10, precision)
    simB, _ = gpu_wave(case, 5, precision)
    blob = simB.checkpoint()
    simC, _ = gpu_wave(case, 0, precision)
    simC.restore(blob)
    assert simC.step_count == 5
    simC.step(5)
    u, v, a = simC.get_state()
    for x, y in zip((u, v, a), gotA[10]):
        assert np.array_equal(x, y)


def test_set_state_roundtrip_and_device_pointers():
    import torch
    sim = _sim((10, 9, 8), 2)
    s = ora.Space((10, 9, 8), 2)
    rng = np.random.default_rng(0)
    u, v, a = (s.pad(rng.standard_normal(s.shape)) for _ in range(3))
    sim.set_state(u, v, a)
    gu, gv, ga = sim.get_state()
    for x, y in ((gu, u), (gv, v), (ga, a)):
        assert rel_l2(x, y) < 1e-14
    tu, tv = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
    sim.set_state(tu, tv)            # a computed as M^{-1}(F - K u)
    ga2 = sim.get_state()[2]
    ref = s.pad(s.pwave_accel(s.interior(u)))
    assert_parity(ga2, ref, 1e-12, "consistent a")
    out = torch.zeros_like(tu)
    sim.get_state_device(u=out)
    assert rel_l2(out.cpu().numpy(), u) < 1e-14


@pytest.fixture(scope="module")
def full_size_reference():
    """Oracle at the full benchmark size: 128^3 elements, p = 2 and 3,
    tau = 2e-3, Ricker x Gaussian (sigma = 0.02) source, 200 steps."""
    out = {}
    for p in (2, 3):
        case = wl.ricker_case(ne=128, p=p)
        out[p] = (case, oracle_wave(case, 200, checkpoints=(10,)))
    return out


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_128cubed_200_steps(full_size_reference, p, precision):
    """The benchmark workload, in the launch configuration the benchmark
    times (graph-replayed steps, default tiles), against the full oracle."""
    case, ref = full_size_reference[p]
    _, got = gpu_wave(case, 200, precision, checkpoints=(10,))
    if precision == "fp64":
        check_state(got[10], ref[10], precision, case.tau, 1e-12, "fp64 p=%d step 10" % p)
        check_state(got[200], ref[200], precision, case.tau, 2e-11, "fp64 p=%d step 200" % p)
    else:
        for n in (10, 200):
            check_state(got[n], ref[n], precision, case.tau, 1e-5, "fp32 p=%d step %d" % (p, n))
    print("p=%d %s rel-L2 u at 200: %.3e" % (p, precision, rel_l2(got[200][0], ref[200][0])))
