"""Per-site Pauli weights and the spreading observables (Sec. 6.4 n(r, t),
Appendix A.3 R_L1, R_L2, S_frac) on the GPU against the oracle.

* The initial network: the observable alone (n = 1 there, 0 elsewhere).
* A 3x3 evolution (FP64 and FP32): the GPU's weights from its converged
  environment against the oracle's weights from its own run of the same
  configuration (bounds 1e-8 / 1e-5).
* A centred observable on 5x5, three steps below chi_max (no truncation,
  and the ZZ bond gates commute, so the colour order cannot break the
  symmetry): C4-symmetric n(r) (Sec. 6.4) within the FP32 bound.
* The radii and the entropy fraction from the library's binding equal the
  oracle's formulas on the same map.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import bp as obp
from oracle import run as oracle_run
from tests.gpu_common import oracle_cfg

pytestmark = pytest.mark.gpu


def test_initial_weights_are_the_observable():
    cfg = pkg.Config(Lx=4, Ly=3, obs=(2, 1), chi_max=4, precision="fp32")
    eng = pkg.Engine(cfg)
    try:
        eng.bp_converge()
        eng.correlator()
        w = eng.pauli_weights()
        sp = eng.spatial()
    finally:
        eng.close()
    want = np.zeros((3, 4, 4))
    want[..., 0] = 1.0
    want[1, 2] = [0, 0, 0, 1]
    assert np.allclose(w, want, atol=1e-12)
    assert sp["R_L1"] == 0.0 and sp["S_frac"] == 0.0


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 1e-5)])
def test_weights_match_the_oracle(prec, tol):
    cfg = pkg.Config(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=8, precision=prec,
                     bp_tol=1e-10 if prec == "fp64" else 1e-7)
    eng = pkg.Engine(cfg)
    try:
        eng.run(8)
        w = eng.pauli_weights().reshape(9, 4)
        sp = eng.spatial()
    finally:
        eng.close()
    _, net = oracle_run.simulate(oracle_cfg(cfg), nsteps=8)
    ref = obp.pauli_weights(net, net.M)
    assert np.max(np.abs(w - ref)) < tol, np.max(np.abs(w - ref))
    n = 1.0 - w[:, 0]
    assert np.max(n) > 1e-3
    so = obp.spatial_observables(n, 3, 3, (1, 1))
    for k in ("R_L1", "R_L2", "S_frac"):
        assert abs(sp[k] - so[k]) < 1e-12, k


def test_centred_weights_are_c4_symmetric():
    cfg = pkg.Config(Lx=5, Ly=5, J=1.0, h=1.5, dt=0.05, order=2, chi_max=16, precision="fp32", bp_tol=1e-7)
    eng = pkg.Engine(cfg)
    try:
        eng.run(3)
        n = 1.0 - eng.pauli_weights()[..., 0]
    finally:
        eng.close()
    for k in range(1, 4):
        assert np.max(np.abs(np.rot90(n, k) - n)) < 1e-5
    assert n[2, 2] > 0.5 and n[1, 2] > 1e-4
