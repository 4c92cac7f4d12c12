"""Pins for the PEPO oracle (oracle/pepo.py, oracle/bp.py, oracle/contract.py).

Expected values come from the dense brute force (itself pinned by closed forms
and free fermions), from closed forms, and from the free-fermion chain.
"""
import numpy as np
import pytest

from oracle import contract, dense, run
from oracle.pepo import Network, bond_key
from tests.free_fermion import autocorrelation_zzx_edge

EXACT = dict(chi_max=10 ** 6, eps_cut=1e-13, bp_alpha=1.0, bp_tol=1e-13, bp_max_sweeps=200)


def test_initial_network_contracts_to_observable():
    net = Network(3, 3, (1, 1), "Z")
    assert np.allclose(contract.to_dense(net), dense.observable(9, 4, "Z"), atol=0)
    assert abs(contract.pinned_value(net) - 1.0) < 1e-15


@pytest.mark.parametrize("gateset,order", [("ZZ_X", 1), ("XX_Z", 2)])
def test_3x3_without_truncation_is_the_dense_operator(gateset, order):
    # Gate/QR/SVD/absorb/deabsorb machinery on a loopy network: with nothing
    # truncated the network must contract to the exact Trotter-evolved operator.
    cfg = dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=order, gateset=gateset, **EXACT)
    c = run.full_config(cfg)
    net = Network(3, 3, c["obs"])
    d = dense.evolve(3, 3, 1.0, 1.0, 0.05, order, 3, c["obs"], gateset=gateset)
    for step in range(1, 4):
        ge = run.trotter_step(net, c)
        assert ge < 1e-20
        dd = dense.evolve(3, 3, 1.0, 1.0, 0.05, order, step, c["obs"], gateset=gateset)
        assert np.max(np.abs(contract.to_dense(net) - dd["O"])) < 1e-8
        assert abs(contract.pinned_value(net) - d["C"][step]) < 1e-10


@pytest.mark.parametrize("order", [1, 2])
def test_chain_bethe_equals_free_fermions(order):
    # BP is exact on a tree (1 x N chain): the Bethe C(t) must equal the exact C(t).
    N, J, h, dt, n = 6, 1.0, 0.7, 0.1, 8
    cfg = dict(Lx=N, Ly=1, J=J, h=h, dt=dt, order=order, obs=(0, 0), **EXACT)
    out, _ = run.simulate(cfg, nsteps=n)
    ff = autocorrelation_zzx_edge(N, J, h, dt, order, n)
    C = np.array([r["C"] for r in out])
    assert np.max(np.abs(C - ff)) < 1e-9
    assert max(abs(r["norm"] - 1.0) for r in out) < 1e-9


def test_chain_interior_observable_bethe_equals_dense():
    N, n = 5, 6
    cfg = dict(Lx=1, Ly=N, J=0.9, h=1.4, dt=0.1, order=2, obs=(0, 2), **EXACT)
    out, _ = run.simulate(cfg, nsteps=n)
    d = dense.evolve(1, N, 0.9, 1.4, 0.1, 2, n, (0, 2))
    C = np.array([r["C"] for r in out])
    assert np.max(np.abs(C - d["C"])) < 1e-9


def test_chain_gate_time_lambda_are_operator_schmidt_values():
    # On a chain with exact (BP-converged) environments the normalised singular
    # values at every gate are the operator-Schmidt values of the evolved
    # operator across that bond.
    N, J, h, dt, n = 6, 1.0, 0.8, 0.1, 4
    cfg = dict(Lx=N, Ly=1, J=J, h=h, dt=dt, order=1, obs=(2, 0), **EXACT)
    c = run.full_config(cfg)
    want = []
    dense.evolve(N, 1, J, h, dt, 1, n, (2, 0),
                 on_bond=lambda s, v1, v2, O: want.append(dense.operator_schmidt_values(O, N, v2)))
    net = Network(N, 1, (2, 0))
    got = []
    for step in range(n):
        rec = []
        run.trotter_step(net, c, rec)
        got.extend(r["lam"] for (_, _, r) in rec)
        run.measure(net, c)
    assert len(got) == len(want)
    for g, w in zip(got, want):
        k = min(len(g), len(w))
        assert np.max(np.abs(g[:k] - w[:k])) < 1e-9
        # anything beyond the common length is a numerical zero on both sides
        assert np.all(g[k:] < 1e-11) and np.all(w[k:] < 1e-11)
        assert np.sum(w > 1e-9) <= len(g)


@pytest.mark.parametrize("gateset,pauli", [("ZZ_X", "X"), ("XX_Z", "Z")])
def test_star_tree_sign_tracking(gateset, pauli):
    # h = 0, observable anticommuting with the bond Pauli at an edge site: the
    # operator spreads only onto its three neighbours (a star, i.e. a tree), so
    # the Bethe value is exact: C(t) = cos(2 J t)^3, negative on (pi/4, 3 pi/4).
    J, dt, n = 1.0, 0.1, 12
    cfg = dict(Lx=3, Ly=3, J=J, h=0.0, dt=dt, order=1, obs=(1, 0), obs_pauli=pauli,
               gateset=gateset, chi_max=16, eps_cut=1e-12, bp_alpha=0.5, bp_tol=1e-13,
               bp_max_sweeps=200)
    out, _ = run.simulate(cfg, nsteps=n)
    C = np.array([r["C"] for r in out])
    ref = np.cos(2 * J * np.arange(n + 1) * dt) ** 3
    assert ref.min() < -0.1
    assert np.max(np.abs(C - ref)) < 1e-10


def test_zzx_J0_pipeline_stays_product_and_gives_cos():
    cfg = dict(Lx=3, Ly=3, J=0.0, h=1.1, dt=0.05, order=1, chi_max=8, bp_tol=1e-12)
    out, net = run.simulate(cfg, nsteps=10)
    C = np.array([r["C"] for r in out])
    assert np.max(np.abs(C - np.cos(2 * 1.1 * np.arange(11) * 0.05))) < 1e-12
    assert all(net.chi(a, b) == 1 for (a, b) in net.lam)


def test_zzx_h0_pipeline_is_one():
    cfg = dict(Lx=3, Ly=3, J=1.0, h=0.0, dt=0.05, order=1, chi_max=8, bp_tol=1e-12)
    out, _ = run.simulate(cfg, nsteps=8)
    assert max(abs(r["C"] - 1.0) for r in out) < 1e-12


def test_truncation_rule_and_lambda_normalisation():
    # Eq. 11 / Eq. 12: chi_new <= chi_max and sum lam^2 = 1 on every bond.
    cfg = dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=3, bp_tol=1e-8)
    out, net = run.simulate(cfg, nsteps=5)
    for r in out[1:]:
        for b, lam in r["lam"].items():
            assert 1 <= len(lam) <= 3
            assert abs(np.sum(lam ** 2) - 1.0) < 1e-12
            assert np.all(np.diff(lam) <= 0)
    assert out[-1]["gate_err"] > 0
