"""ads_apply_noalloc: the operators of ads_apply for callers that cannot
allocate device memory during the call (a host application whose device
memory is all handed out up front, or a loop that cannot take the
synchronisation cudaMalloc may cost).  The entry point uses a fixed scratch
array compiled into the library.

Checked through the C ABI, on two calls in a row for every operator (the
fixed scratch keeps the previous call's contents):
  - against the oracle's operators (mass, stiffness, mass solve, split
    solve), element-wise within the FP64 operator tolerance of the other
    tests (1e-12 relative L2);
  - against ads_apply on the same input, within the same tolerance;
  - the call reaches the simulation's allocator zero times (ads_apply, the
    control, reaches it);
  - on FP64 and FP32 simulations (the operators are FP64 on both).
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle as ora
from tests.cases import assert_parity

pytestmark = pytest.mark.gpu

OPS = (0, 1, 2, 3)   # ADS_OP_MASS, ADS_OP_STIFF, ADS_OP_MASS_SOLVE, ADS_OP_SPLIT_SOLVE
TOL = 1e-12


def _oracle_ops(s, x, tau):
    eta = tau * tau / 4
    return {0: s.apply_mass(x), 1: s.apply_lap(x), 2: s.solve_mass(x), 3: s.solve_kron((eta, eta, eta), x)}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ne,p", [((20, 18, 16), 2), ((11, 13, 9), 3)])
def test_noalloc_matches_oracle_and_apply_twice(ne, p, precision, monkeypatch):
    import torch
    from paper_1911_08158_gb300 import Simulation
    tau = 0.02
    sim = Simulation(ne, p, tau, precision=precision)
    s = ora.Space(ne, p)
    # every device allocation of the library goes through this simulation's
    # allocator callback, which calls torch.cuda.caching_allocator_alloc
    calls = {"n": 0}
    real_alloc = torch.cuda.caching_allocator_alloc

    def counting_alloc(*a, **k):
        calls["n"] += 1
        return real_alloc(*a, **k)

    monkeypatch.setattr(torch.cuda, "caching_allocator_alloc", counting_alloc)
    rng = np.random.default_rng(11 + p)
    for op in OPS:
        for call in range(2):
            x = rng.standard_normal(s.shape)
            ref = s.pad(_oracle_ops(s, x, tau)[op])
            xf = s.pad(x)
            n0 = calls["n"]
            via_apply = sim.apply(op, xf)
            assert calls["n"] > n0, "control: ads_apply should reach the allocator"
            xd = torch.tensor(xf, device="cuda")
            out = torch.full_like(xd, float("nan"))
            torch.cuda.synchronize()
            n0 = calls["n"]
            sim.apply_noalloc(op, xd, out)
            assert calls["n"] == n0, "ads_apply_noalloc reached the allocator"
            got = out.cpu().numpy()
            assert_parity(got, ref, TOL, "%s op %d call %d vs oracle" % (precision, op, call))
            assert_parity(got, via_apply, TOL, "%s op %d call %d vs ads_apply" % (precision, op, call))
            # boundary coefficients are written as zero
            assert np.all(got[0] == 0) and np.all(got[:, -1] == 0) and np.all(got[..., 0] == 0)


def test_noalloc_rejects_spaces_beyond_its_scratch():
    import torch
    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation((100, 80, 80), 2, 0.02, precision="fp64")   # 102*80*80 padded interior > 524288
    xd = torch.zeros(sim.n[::-1], dtype=torch.float64, device="cuda")
    with pytest.raises(ads.AdsError) as e:
        sim.apply_noalloc(0, xd, torch.zeros_like(xd))
    assert e.value.code == -5


def test_noalloc_rejects_host_memory_through_the_c_abi():
    """Pointers that are not device memory of the simulation's device are
    refused on the host, before any work is queued."""
    import torch
    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation((8, 9, 10), 2, 0.02, precision="fp64")
    n = sim.count
    host = np.zeros(n)
    dev = torch.zeros(n, dtype=torch.float64, device="cuda")
    lib = ads.library()
    assert lib.ads_apply_noalloc(sim.handle, 0, host.ctypes.data, dev.data_ptr(), n) == -1
    assert lib.ads_apply_noalloc(sim.handle, 0, dev.data_ptr(), host.ctypes.data, n) == -1
    assert lib.ads_apply_noalloc(sim.handle, 0, dev.data_ptr(), dev.data_ptr(), n + 1) == -1
