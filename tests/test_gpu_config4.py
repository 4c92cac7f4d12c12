"""Config 4 (8x8, J = 1, h = 2, Z at (3, 3), second-order split, dt = 0.05,
chi_max = 64) on the GPU in all three precisions against the oracle's
trajectory prefix (tests/golden/traj_c4_chi64.txt, written by
tests/golden/make_trajectories.py, which calls only the oracle; the oracle
needs minutes per step from t = 0.3 on, so the file holds the prefix it
finished).

Bounds per compared layer: |dC| <= 1e-8 (FP64), 1e-5 (FP32), 1e-3 (split
TF32), plus d * bp_tol where the single-layer sweep counts differ by d (the
Eq. 14 stopping rule, as in the config-2 test); trapped layers are handled
by the config-2 rule; flags bit 0 clear.  Over these layers the bonds grow
from 1 to chi_max at the centre, so every QR branch and the truncation are
exercised: the Eq. 10 rule sends every site to Householder while n <= 150,
then Cholesky-QR sites appear and most of them fail the Gram trust test.
"""
import os

import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from tests.gpu_common import gpu_run
from tests.test_gpu_config2 import BP_TOL, compared_steps

pytestmark = pytest.mark.gpu

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "traj_c4_chi64.txt")
TOL = {"fp64": 1e-8, "fp32": 1e-5, "tf32x3": 1e-3}


def load():
    C, sw2, sw1 = [], [], []
    with open(PATH) as f:
        for line in f:
            p = line.split()
            if line.startswith("# config"):
                assert "bp_tol=%g" % BP_TOL in p, line
            if not p or p[0].startswith("#") or p[0] == "lam":
                continue
            assert int(p[0]) == len(C)
            C.append(float(p[2]))
            sw2.append(int(p[5]))
            sw1.append(int(p[6]))
    return np.array(C), np.array(sw2), np.array(sw1)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_config4_prefix_matches_the_oracle(prec):
    Cref, sw2r, sw1r = load()
    n = len(Cref) - 1
    assert n >= 5
    cfg = pkg.Config(Lx=8, Ly=8, J=1.0, h=2.0, dt=0.05, order=2, obs=(3, 3), chi_max=64, precision=prec)
    recs, _ = gpu_run(cfg, n)
    C = np.array([r["C"] for r in recs])
    sw2 = np.array([r["bp_sweeps"] for r in recs])
    sw1 = np.array([r["bp1_sweeps"] for r in recs])
    keep, skipped = compared_steps(sw2, sw1, sw2r, sw1r)
    assert len(keep) >= 5
    bound = TOL[prec] + np.abs(sw1 - sw1r)[keep] * BP_TOL
    err = np.abs(C[keep] - Cref[keep])
    print("config 4 %s: %d layers, %d compared, max |dC| = %.3g" % (prec, n, len(keep), float(np.max(err))))
    assert np.all(err < bound), [(keep[i], float(err[i]), float(bound[i])) for i in np.nonzero(err >= bound)[0]]
    flags = 0
    for r in recs:
        flags |= int(r["flags"])
    assert flags & 1 == 0
