"""The CSV regenerator of the paper's experiments (energy histories and
second order in time, Sec. 4 and Sec. 6), at reduced size."""
import csv
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _read(path):
    with open(path) as f:
        r = list(csv.reader(f))
    return r[0], np.array([[float(v) for v in row] for row in r[1:]])


def test_experiment_tables(tmp_path):
    from paper_1911_08158_gb300.experiments import run_all
    run_all(str(tmp_path), quick=True)
    for kind in ("pwave", "elastic"):
        h, E = _read(os.path.join(tmp_path, "%s_energies.csv" % kind))
        assert h == ["step", "t", "kinetic", "potential", "total", "invariant"]
        inv = E[:, 5]
        assert np.all(E[:, 2] >= 0) and np.all(E[:, 3] >= -1e-15)
        # the scheme's invariant is constant from the first step on
        assert np.abs(inv[1:] - inv[1]).max() <= 1e-10 * abs(inv[1]), kind
        # energy moves between kinetic and potential
        assert E[:, 2].max() > 2 * E[:, 2].min() + 1e-30
        h, O = _read(os.path.join(tmp_path, "%s_time_order.csv" % kind))
        assert h == ["tau", "rel_l2_error", "observed_order"]
        assert np.all(np.diff(O[:, 1]) < 0)                 # errors fall as tau halves
        assert 1.7 <= O[-1, 2] <= 2.4, (kind, O)            # second order (Sec. 4, Sec. 6)
