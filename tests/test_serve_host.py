"""Host logic of the continuous-batching loop, with fake simulations and a
simulated clock (no GPU): admission by budget in arrival order, state kept
until completion, every request run for exactly its steps, latencies from
arrival to result."""
import numpy as np

from paper_1911_08158_gb300 import workloads as wl
from paper_1911_08158_gb300.serve import Server, request_dofs


class FakeSim:
    def __init__(self, req):
        self.req = req
        self.steps = 0
        self.closed = False


class World:
    """Simulated time: a batch call of k steps costs k * (sum of member DOFs) * rate."""

    def __init__(self, rate=1e-9):
        self.t = 0.0
        self.rate = rate
        self.calls = []
        self.live = set()

    def clock(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)

    def batch(self, sims, k):
        assert len({id(s) for s in sims}) == len(sims)
        assert all(not s.closed for s in sims)
        self.calls.append((len(sims), k))
        for s in sims:
            s.steps += k
            assert s.steps <= s.req.steps
        self.t += k * sum(request_dofs(s.req) for s in sims) * self.rate

    def factory(self, req):
        s = FakeSim(req)
        self.live.add(id(s))
        return s

    def close(self, s):
        s.closed = True
        self.live.discard(id(s))


def _server(world, budget, **kw):
    est = lambda r: request_dofs(r) * 16   # noqa: E731
    return Server(budget, factory=world.factory, batch=world.batch, estimate=est,
                  fetch=lambda s: s.steps, close=world.close, clock=world.clock, sleep=world.sleep,
                  keep_state=True, **kw)


def test_every_request_completes_with_its_steps():
    reqs = wl.serving_requests(count=120, rate=50.0, seed=3, lo=8, hi=40, max_steps=60)
    w = World()
    rep = _server(w, budget=10 ** 12).run(reqs)
    assert len(rep.results) == 120 and not rep.rejected
    for r in reqs:
        res = rep.results[r.rid]
        assert res.state == r.steps            # the fake's step count at completion
        assert res.done >= res.admitted >= r.arrival - 1e-12
        assert res.latency >= 0
    assert not w.live


def test_budget_is_never_exceeded_and_admission_is_fifo():
    reqs = wl.serving_requests(count=80, rate=400.0, seed=5, lo=8, hi=48, max_steps=80)
    est = {r.rid: request_dofs(r) * 16 for r in reqs}
    budget = int(np.percentile(list(est.values()), 90) * 3)
    w = World(rate=1e-8)
    order = []
    inner = w.factory

    def factory(r):
        order.append(r.rid)
        # resident bytes of the live set, including this one, stay within budget
        live_bytes = sum(est[s] for s in live_ids) + est[r.rid]
        assert live_bytes <= budget
        live_ids.add(r.rid)
        return inner(r)

    live_ids = set()

    def close(s):
        live_ids.discard(s.req.rid)
        w.close(s)

    srv = _server(w, budget)
    srv.factory, srv.close = factory, close
    rep = srv.run(reqs)
    admitted = [r.rid for r in sorted(reqs, key=lambda r: (r.arrival, r.rid)) if r.rid not in rep.rejected]
    assert order == admitted                          # arrival order
    assert rep.peak_bytes <= budget
    assert set(rep.rejected) == {r.rid for r in reqs if est[r.rid] > budget}
    assert rep.max_live > 1                           # requests overlap


def test_calls_stop_at_the_nearest_completion():
    reqs = [wl.Request(0, 0.0, "wave", (8, 8, 8), 2, 1e-3, 10, {}),
            wl.Request(1, 0.0, "wave", (8, 8, 8), 2, 1e-3, 25, {}),
            wl.Request(2, 0.0, "elastic", (8, 8, 8), 2, 1e-3, 7, {})]
    w = World()
    rep = _server(w, budget=10 ** 12, chunk=16).run(reqs)
    assert w.calls == [(3, 7), (2, 3), (1, 15)]
    assert [rep.results[i].state for i in range(3)] == [10, 25, 7]
    s = rep.summary()
    assert s["requests"] == 3 and s["p99_s"] >= s["p50_s"] >= 0
