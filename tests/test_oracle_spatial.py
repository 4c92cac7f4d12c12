"""Pins of the oracle's per-site Pauli weights (Sec. 6.4 n(r, t), Appendix
A.3 radii and spatial entropy).

* The initial network (Sec. 2.3): the observable Pauli at its site, the
  identity everywhere else, so n(r) is 1 at the observable and 0 elsewhere.
* Chains are trees, where BP is exact: after untruncated Trotter steps the
  weights from the BP environment equal the weights of the dense Trotter-
  evolved operator, O = sum_p P_p (x) B_p at each site, computed by partial
  traces (an independent method).  One bond is first regauged by a
  non-orthogonal X X^-1 (the operator is unchanged, the two messages of
  that bond then differ), so the pin also fixes which message of a bond
  belongs to which site.
* A centred observable on a 3x3 grid: the weights in the converged BP
  environment are C4-symmetric (the paper's exact four-fold symmetry of
  n(r, t), Sec. 6.4), although the colour order breaks the symmetry of the
  individual bond updates.
* The radii and the entropy fraction of a weight map concentrated on one
  site are 0; of a uniform map, S_frac = 1.
"""
import numpy as np

from oracle import bp as obp
from oracle import dense
from oracle.pepo import Network, leg_apply
from oracle.run import full_config, measure, trotter_step


def test_initial_network_is_the_observable_alone():
    net = Network(3, 3, (1, 1), "Z")
    w = obp.pauli_weights(net, net.M)
    want = np.zeros((9, 4))
    want[:, 0] = 1.0
    want[4] = [0, 0, 0, 1]
    assert np.allclose(w, want, atol=1e-15)
    n = 1.0 - w[:, 0]
    s = obp.spatial_observables(n, 3, 3, (1, 1))
    assert s["R_L1"] == 0.0 and s["R_L2"] == 0.0 and s["S_frac"] == 0.0


def test_uniform_map_has_unit_entropy_fraction():
    s = obp.spatial_observables(np.ones(16), 4, 4, (1, 1))
    assert abs(s["S_frac"] - 1.0) < 1e-15
    # mean Manhattan distance from (1, 1) over the 4x4 grid: (1+0+1+2)/4 * 2
    assert abs(s["R_L1"] - 2.0) < 1e-15


def test_chain_weights_equal_the_dense_operator():
    N, nsteps = 6, 4
    cfg = full_config(dict(Lx=N, Ly=1, J=1.0, h=0.7, dt=0.1, order=2, obs=(2, 0), chi_max=64, eps_cut=0.0,
                           bp_alpha=1.0, bp_tol=1e-14, bp_max_sweeps=200))
    net = Network(N, 1, cfg["obs"], "Z")
    for _ in range(nsteps):
        trotter_step(net, cfg)
    a, b = 2, 3
    ka, kb = net.axis(a, b), net.axis(b, a)
    chi = net.O[a].shape[ka]
    X = np.eye(chi) + 0.4 * np.random.default_rng(5).standard_normal((chi, chi))
    net.O[a] = leg_apply(net.O[a], ka, X.T)
    net.O[b] = leg_apply(net.O[b], kb, np.linalg.inv(X))
    measure(net, cfg)
    assert np.max(np.abs(net.M[(a, b)] - net.M[(b, a)])) > 1e-2
    w = obp.pauli_weights(net, net.M)
    ref = dense.site_pauli_weights(dense.evolve(N, 1, 1.0, 0.7, 0.1, 2, nsteps, (2, 0))["O"], N)
    assert np.max(np.abs(w - ref)) < 1e-10, np.max(np.abs(w - ref))
    assert np.max(1.0 - ref[:, 0]) > 0.05     # the operator has spread


def test_centred_observable_gives_c4_symmetric_weights():
    cfg = full_config(dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.1, order=2, obs=(1, 1), chi_max=16, eps_cut=0.0,
                           bp_alpha=0.5, bp_tol=1e-12, bp_max_sweeps=300))
    net = Network(3, 3, (1, 1), "Z")
    trotter_step(net, cfg)
    measure(net, cfg)
    n = (1.0 - obp.pauli_weights(net, net.M)[:, 0]).reshape(3, 3)
    for k in range(1, 4):
        assert np.max(np.abs(np.rot90(n, k) - n)) < 1e-8
    assert n[0, 1] > 1e-6 and n[1, 1] > 0.5     # the edge sites are reached after one step
