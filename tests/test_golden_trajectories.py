"""Provenance of the stored oracle trajectories (tests/golden/traj_*.txt).

Each file was written by tests/golden/make_trajectories.py, which calls only
the oracle.  Here the oracle is run again, on the CPU, for the first steps
of every stored case (the cheap ones: bonds still small), and the stored
lines must match: the configuration header exactly, C, C_proj and the BP
sweep counts to rounding.  A stored value that did not come from this
oracle, or an oracle changed since the files were written, fails here.
"""
import os

import numpy as np
import pytest

from oracle.pepo import Network
from oracle.run import full_config, measure, trotter_step
from tests.golden.make_trajectories import CASES

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STEPS = 3


def stored(name):
    head, rows = None, []
    with open(os.path.join(HERE, "traj_%s.txt" % name)) as f:
        for line in f:
            if line.startswith("# config "):
                head = line[len("# config "):].strip()
            elif line.strip() and not line.startswith("#") and not line.startswith("lam"):
                p = line.split()
                rows.append((int(p[0]), float(p[2]), float(p[3]), int(p[5]), int(p[6])))
    return head, rows


@pytest.mark.parametrize("name", sorted(CASES))
def test_stored_trajectory_prefix_is_the_oracle(name):
    head, rows = stored(name)
    case = dict(CASES[name])
    case.pop("nsteps")
    c = full_config(case)
    assert head == " ".join("%s=%s" % (k, c[k]) for k in sorted(c) if k != "nsteps")
    net = Network(c["Lx"], c["Ly"], c["obs"], c["obs_pauli"])
    for step in range(STEPS + 1):
        if step > 0:
            trotter_step(net, c)
        r = measure(net, c)
        s, C, Cp, sw2, sw1 = rows[step]
        assert s == step
        assert abs(r["C"] - C) < 1e-12 and abs(r["C_proj"] - Cp) < 1e-12, (name, step, r["C"], C)
        assert (r["bp_sweeps"], r["bp1_sweeps"]) == (sw2, sw1), (name, step)
