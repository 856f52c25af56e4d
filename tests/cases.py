"""Run a seeded workload through the oracle and through the CUDA library.
Both sides take the same parameters from paper_1911_08158_gb300.workloads."""
import numpy as np

import oracle as ora


def oracle_wave(case, steps, checkpoints=(), boundary="dirichlet"):
    """Returns {step: (u, v, a)} (full arrays) at the requested steps."""
    s = ora.Space(case.n_elem, case.p, natural=boundary == "natural")
    G, rick = None, (8.0, 0.125)
    if case.source:
        src = case.source
        G = s.load_gauss(src["amp"], src["center"], src["den"])
        rick = (src["freq"], src["t0"])
    if case.u0:
        u = s.project_gauss(case.u0["amp"], case.u0["center"], case.u0["den"])
    else:
        u = s.zeros()
    v = s.zeros()
    a = s.pwave_accel(u, 0.0, case.c2, G, rick)
    out = {}
    done = 0
    for target in sorted(set(checkpoints) | {steps}):
        u, v, a = s.pwave_run(u, v, a, case.tau, target - done, step0=done, c2=case.c2, G=G, rick=rick)
        done = target
        out[target] = (s.pad(u), s.pad(v), s.pad(a))
    return out


def gpu_wave(case, steps, precision="fp64", checkpoints=(), **kw):
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, c2=case.c2, precision=precision, **kw)
    if case.source:
        sim.set_source(case.source)
    sim.set_gaussian_state(case.u0, None)
    out = {}
    done = 0
    for target in sorted(set(checkpoints) | {steps}):
        sim.step(target - done)
        done = target
        out[target] = sim.get_state()
    return sim, out


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def assert_parity(got, ref, tol, what=""):
    """Element-wise comparison: relative L2 over the whole field within tol,
    and every element within 10*tol of the field's max magnitude."""
    r = rel_l2(got, ref)
    scale = max(np.abs(ref).max(), 1e-300)
    emax = float(np.abs(got - ref).max() / scale)
    assert r <= tol and emax <= 10 * tol, "%s: rel-L2 %.3e, max elem err %.3e (tol %.1e)" % (what, r, emax, tol)
    return r


def derived_tols(u, v, a, tau, base):
    """Tolerances for v and a given the displacement tolerance `base`.

    Rounding noise in the displacement is white: it populates every mode up
    to the highest frequency the implicit Newmark scheme represents, 2/tau
    (modes with omega*tau >> 1 advance by ~pi per step).  Differencing it in
    time scales it by 2/tau for the velocity and (2/tau)^2 for the
    acceleration, so relative to the fields themselves
        tol_v = base * (2/tau) |u| / |v|,   tol_a = base * (2/tau)^2 |u| / |a|,
    never tighter than `base`."""
    nu, nv, na = (max(float(np.linalg.norm(x)), 1e-300) for x in (u, v, a))
    w = 2.0 / tau
    return max(base, base * w * nu / nv), max(base, base * w * w * nu / na)


def check_state(got, ref, precision, tau, base, what=""):
    """u within `base` (the displacement is the solution the tolerance is
    stated for); v and a within the derived tolerances above."""
    assert_parity(got[0], ref[0], base, what + " u")
    tv, ta = derived_tols(ref[0], ref[1], ref[2], tau, base)
    assert_parity(got[1], ref[1], tv, what + " v (tol %.1e)" % tv)
    assert_parity(got[2], ref[2], ta, what + " a (tol %.1e)" % ta)


def oracle_elastic(case, steps, checkpoints=(), source=None, boundary="dirichlet"):
    """Returns {step: (U, V)} with V = (U^n - U^{n-1})/tau (full arrays)."""
    s = ora.Space(case.n_elem, case.p, natural=boundary == "natural")
    V0 = np.zeros((3,) + s.shape)
    if case.v0:
        g = s.project_gauss(case.v0["amp"], case.v0["center"], case.v0["den"])
        V0 = np.stack([case.v0["dir"][i] * g for i in range(3)])
    U0 = np.zeros_like(V0)
    kw = {}
    if source:
        G = s.load_gauss(source["amp"], source["center"], source["den"])
        kw = dict(G=G, direction=np.asarray(source["dir"], float), rick=(source["freq"], source["t0"]))
    Up = s.elastic_start(case.tau, case.lam, case.mu, case.rho, U0, V0, **kw, **({"t0": 0.0} if kw else {}))
    out, done, U = {}, 0, U0
    for target in sorted(set(checkpoints) | {steps}):
        U, Up = s.elastic_run(case.tau, case.lam, case.mu, case.rho, target - done, U, Up, step0=done, **kw)
        done = target
        out[target] = (s.pad(U), s.pad((U - Up) / case.tau))
    return out


def gpu_elastic(case, steps, precision="fp64", checkpoints=(), source=None, boundary="dirichlet"):
    from paper_1911_08158_gb300 import Simulation
    sim = Simulation(case.n_elem, case.p, case.tau, kind="elastic", lam=case.lam, mu=case.mu, rho=case.rho,
                     precision=precision, boundary=boundary)
    if source:
        sim.set_source(source)
    sim.set_gaussian_state(None, case.v0)
    out, done = {}, 0
    for target in sorted(set(checkpoints) | {steps}):
        sim.step(target - done)
        done = target
        out[target] = sim.get_state()[:2]
    return sim, out
