"""Config 2 as configured: the 4x4 grid, J = 1, h = 2, Z at (1, 1) (off
centre), second-order split, dt = 0.05, 40 steps (t = 2), chi_max in
{20, 40, 60}: the FP32 GPU path (and the split-TF32 tensor-core mode) against
the oracle's trajectories, stored by tests/golden/make_trajectories.py (which
calls only the oracle; the chi_max = 60 file holds the prefix the oracle
finished, the run taking many hours on the host).

Bounds: |dC| <= 1e-5 (FP32), 1e-3 (split TF32) at every stored step; the
Vidal spectra after the last step (when stored) within 1e-5 / 1e-4 of
lam_0; flags bit 0 clear (no rank-deficient message, where the GPU's Q-less
update would depart from the literal one).
"""
import os

import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from tests.gpu_common import gpu_run, lam_errors

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"fp32": (1e-5, 1e-5), "tf32x3": (1e-3, 1e-4)}


def load(chi):
    path = os.path.join(HERE, "traj_c2_chi%d.txt" % chi)
    C, lam = [], {}
    with open(path) as f:
        for line in f:
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] == "lam":
                lam[int(p[1])] = np.array([float(x) for x in p[3:]])
            else:
                assert int(p[0]) == len(C)
                C.append(float(p[2]))
    return np.array(C), lam


@pytest.mark.parametrize("chi", [20, 40, 60])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_config2_trajectory(chi, prec):
    Cref, lref = load(chi)
    n = len(Cref) - 1
    assert n >= 10
    cfg = pkg.Config(Lx=4, Ly=4, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=chi, precision=prec)
    recs, lam = gpu_run(cfg, n)
    C = np.array([r["C"] for r in recs])
    dC = float(np.max(np.abs(C - Cref)))
    print("config 2 chi %d %s: %d steps, max |dC| = %.3g" % (chi, prec, n, dC))
    assert dC < TOL[prec][0], dC
    flags = 0
    for r in recs:
        flags |= int(r["flags"])
    assert flags & 1 == 0
    if lref:
        lam_err, _ = lam_errors(lam, lref)
        assert lam_err < TOL[prec][1], lam_err
