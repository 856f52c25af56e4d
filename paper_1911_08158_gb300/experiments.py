"""Regenerate the paper's experiments as CSV tables (headless).

Sec. 4 (scalar P-wave) and Sec. 6 (linear elasticity) run 32^3-element
problems and report (a) the kinetic, potential and total energy over the
run and (b) second-order convergence in time.  This module runs the same
kinds of experiments through the library and writes one CSV per table:

  pwave_energies.csv     step, t, kinetic, potential, total, invariant
  elastic_energies.csv   step, t, kinetic, potential, total, invariant
  pwave_time_order.csv   tau, rel_l2_error, observed_order
  elastic_time_order.csv tau, rel_l2_error, observed_order

Data (the paper leaves degree, initial data and run length open):
Gaussian initial pulses (displacement for the scalar wave, velocity along a
fixed direction for elasticity), homogeneous Dirichlet boundary, no source,
p = 2.  "invariant" is the exactly conserved discrete energy of the scheme;
"total" is kinetic + potential, which the scheme keeps constant up to O(tau^2).
The time-order tables compare each tau with a run at tau / 8 at a common
final time; observed_order is log2 of the error ratio between consecutive
rows (tau halves each row).

    python -m paper_1911_08158_gb300.experiments --out DIR [--quick]
"""
from __future__ import annotations

import argparse
import csv
import math
import os

import numpy as np

PULSE = dict(amp=1.0, center=(0.5, 0.5, 0.5), den=0.01)
VPULSE = dict(amp=1.0, dir=(0.48, 0.6, 0.64), center=(0.5, 0.5, 0.5), den=2 * 0.05 ** 2)


def _write(path, header, rows):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(header)
        for r in rows:
            w.writerow(["%.10g" % v if isinstance(v, float) else v for v in r])


def _wave(ne, p, tau, precision="fp64"):
    from .ads import Simulation
    sim = Simulation(ne, p, tau, precision=precision)
    sim.set_gaussian_state(PULSE, None)
    return sim


def _elastic(ne, p, tau, precision="fp64"):
    from .ads import Simulation
    sim = Simulation(ne, p, tau, kind="elastic", precision=precision)
    sim.set_gaussian_state(None, VPULSE)
    return sim


def energies(kind, ne=32, p=2, tau=0.01, steps=200, every=1, csv_path=None):
    """Energy history of one run: rows (step, t, kinetic, potential, total, invariant)."""
    sim = (_wave if kind == "wave" else _elastic)(ne, p, tau)
    rows = []
    for n in range(0, steps + 1, every):
        if n:
            sim.step(every)
        k, u, inv = sim.energy()
        # scalar wave: the invariant is modified kinetic + potential; elasticity reports it whole
        invariant = inv + u if kind == "wave" else inv
        rows.append((n, n * tau, k, u, k + u, invariant))
    if csv_path:
        _write(csv_path, ["step", "t", "kinetic", "potential", "total", "invariant"], rows)
    return rows


def time_order(kind, ne=16, p=2, T=0.32, taus=(0.04, 0.02, 0.01, 0.005), csv_path=None):
    """Relative L2 error of the displacement at time T for each tau against a
    run at min(tau) / 8; rows (tau, error, observed order)."""
    make = _wave if kind == "wave" else _elastic

    def final(tau):
        sim = make(ne, p, tau)
        sim.step(int(round(T / tau)))
        return sim.get_state(fields=("u",))[0]

    ref = final(min(taus) / 8)
    rows, prev = [], None
    for tau in sorted(taus, reverse=True):
        e = float(np.linalg.norm(final(tau) - ref) / np.linalg.norm(ref))
        order = math.log2(prev / e) if prev else float("nan")
        rows.append((tau, e, order))
        prev = e
    if csv_path:
        _write(csv_path, ["tau", "rel_l2_error", "observed_order"], rows)
    return rows


def run_all(out, quick=False):
    os.makedirs(out, exist_ok=True)
    ne, steps, ne_o = (12, 40, 8) if quick else (32, 200, 16)
    energies("wave", ne=ne, steps=steps, csv_path=os.path.join(out, "pwave_energies.csv"))
    energies("elastic", ne=ne, steps=steps, csv_path=os.path.join(out, "elastic_energies.csv"))
    time_order("wave", ne=ne_o, csv_path=os.path.join(out, "pwave_time_order.csv"))
    time_order("elastic", ne=ne_o, csv_path=os.path.join(out, "elastic_time_order.csv"))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--quick", action="store_true", help="small grids and short runs")
    a = ap.parse_args()
    run_all(a.out, a.quick)


if __name__ == "__main__":
    main()
