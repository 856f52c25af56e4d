"""ads_apply_noalloc: the operators of ads_apply for callers that cannot
allocate device memory at the point of the call (stream capture, fixed
memory budgets).  Through the C ABI, its output must equal ads_apply's within
the FP64 operator tolerance of the other tests (1e-12 relative L2), on two
calls in a row (the fixed scratch keeps the previous call's contents)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OPS = (0, 1, 2, 3)   # ADS_OP_MASS, ADS_OP_STIFF, ADS_OP_MASS_SOLVE, ADS_OP_SPLIT_SOLVE


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


@pytest.mark.parametrize("ne,p", [((20, 18, 16), 2), ((11, 13, 9), 3)])
def test_noalloc_matches_apply_twice(ne, p):
    import torch
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(ne, p, 0.02, precision="fp64")
    rng = np.random.default_rng(11)
    for op in OPS:
        for call in range(2):
            x = rng.standard_normal(sim.n[::-1])
            x[0] = x[-1] = 0.0
            x[:, 0] = x[:, -1] = 0.0
            x[..., 0] = x[..., -1] = 0.0
            ref = sim.apply(op, x)
            xd = torch.tensor(x, device="cuda")
            out = torch.full_like(xd, float("nan"))
            sim.apply_noalloc(op, xd, out)
            got = out.cpu().numpy()
            assert _rel(got, ref) <= 1e-12, (op, call, _rel(got, ref))


def test_noalloc_rejects_spaces_beyond_its_scratch():
    import torch
    import paper_1911_08158_gb300 as ads
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation((100, 80, 80), 2, 0.02, precision="fp64")   # 102*80*80 padded interior > 524288
    xd = torch.zeros(sim.n[::-1], dtype=torch.float64, device="cuda")
    with pytest.raises(ads.AdsError) as e:
        sim.apply_noalloc(0, xd, torch.zeros_like(xd))
    assert e.value.code == -5
