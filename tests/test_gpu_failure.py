"""Failure detection without a GPU fault.

- A device-side wait that runs out: the library's bounded mbarrier wait is
  made to expire on purpose (a barrier whose bytes never arrive); the
  kernel records the timeout and returns, the host gets ADS_ERR_TIMEOUT,
  and the context stays usable for real work afterwards.
- Device allocation failure: an allocator callback that refuses (at once,
  or after some allocations) makes ads_create fail with ADS_ERR_OOM and
  hand back every allocation it had made."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ADS_ERR_OOM, ADS_ERR_TIMEOUT = -2, -4


def test_bounded_wait_times_out_and_context_survives():
    from paper_1911_08158_gb300 import Simulation
    from paper_1911_08158_gb300.ads import selftest_timeout
    from paper_1911_08158_gb300 import workloads as wl
    assert selftest_timeout(0, 20_000_000) == ADS_ERR_TIMEOUT
    c = wl.pulse_case(ne=8, p=2, steps=0)
    s = Simulation(c.n_elem, c.p, c.tau, precision="fp32")
    s.set_gaussian_state(c.u0, None)
    s.step(3)
    u = s.get_state()[0]
    assert np.isfinite(u).all() and np.abs(u).max() > 0


def _create_with(alloc_budget):
    """ads_create with a cudaMalloc-backed allocator that refuses after
    `alloc_budget` allocations; returns (rc, live allocations left)."""
    import torch
    from paper_1911_08158_gb300 import ads as A
    L = A.library()
    live = {}
    count = [0]

    def alloc(nbytes, ctx):
        if count[0] >= alloc_budget:
            return None
        count[0] += 1
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, ctx):
        live.pop(ptr, None)

    fa, ff = A.ALLOC_FN(alloc), A.FREE_FN(free)
    grid = A.Grid((ctypes.c_int * 3)(6, 7, 8), (ctypes.c_double * 3)(1.0, 1.0, 1.0))
    mat = A.Material(A.ADS_SCALAR_WAVE, 1.0, 1.0, 1.0, 1.0)
    opts = A.Options(A.ADS_FP32, 0, None, fa, ff, None, 0, 0)
    h = ctypes.c_void_p()
    rc = L.ads_create(ctypes.byref(grid), 2, 1e-2, ctypes.byref(mat), ctypes.byref(opts), ctypes.byref(h))
    if rc == 0:
        L.ads_destroy(h)
    torch.cuda.synchronize()
    return rc, len(live), count[0]


@pytest.mark.parametrize("budget", [0, 3, 12])
def test_allocator_refusal_reports_oom_and_releases_everything(budget):
    rc, left, made = _create_with(budget)
    assert rc == ADS_ERR_OOM
    assert made == budget and left == 0


def test_allocator_that_never_refuses_creates_and_frees_all():
    rc, left, made = _create_with(10 ** 6)
    assert rc == 0 and made > 12 and left == 0
