"""Continuous batching on the GPU: a Poisson stream of mixed scalar-wave and
elasticity requests served under an HBM budget; each result must be the one
the request gets alone (the grouped launches share no data between members,
so the comparison is exact)."""
import numpy as np
import pytest

from paper_1911_08158_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _stream():
    return wl.serving_requests(count=24, rate=300.0, seed=11, lo=6, hi=28, max_steps=40)


def test_served_results_equal_alone_runs():
    from paper_1911_08158_gb300 import estimate_bytes
    from paper_1911_08158_gb300.serve import Server, make_simulation
    reqs = _stream()
    alone = {}
    for r in reqs:
        s = make_simulation(r, "fp32")
        s.step(r.steps)
        alone[r.rid] = s.get_state(fields=("u",))[0]
        s.close()
    est = [estimate_bytes(r.n_elem, r.p, r.kind, "fp32") for r in reqs]
    budget = int(sorted(est)[-1] * 2.5)       # forces requests to wait for memory
    rep = Server(budget, precision="fp32", chunk=8, keep_state=True).run(reqs)
    assert not rep.rejected and len(rep.results) == len(reqs)
    assert rep.peak_bytes <= budget and rep.max_live > 1
    for r in reqs:
        got = rep.results[r.rid].state
        assert np.array_equal(got, alone[r.rid]), "request %d (%s %s p=%d)" % (r.rid, r.kind, r.n_elem, r.p)
    s = rep.summary()
    assert s["p99_s"] >= s["p50_s"] > 0


def test_estimate_bounds_actual_device_bytes():
    from paper_1911_08158_gb300 import estimate_bytes
    from paper_1911_08158_gb300.serve import make_simulation
    for r in _stream()[:8]:
        for prec in ("fp32", "fp64"):
            s = make_simulation(r, prec)
            actual = s.device_bytes
            est = estimate_bytes(r.n_elem, r.p, r.kind, prec)
            assert actual <= est <= 4 * actual + (64 << 20), (r.kind, r.n_elem, r.p, prec, actual, est)
            s.close()
