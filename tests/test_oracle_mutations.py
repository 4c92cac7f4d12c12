"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one plausible error into the oracle (on the CPU only) and
checks that a pin from test_oracle_dense / test_oracle_pepo then fails; this
shows the pins constrain every part of the oracle they cover.
"""
import numpy as np
import pytest

from oracle import bp as obp
from oracle import contract, dense, gates, pepo, run
from tests.free_fermion import autocorrelation_zzx_edge

EXACT = dict(chi_max=10 ** 6, eps_cut=1e-13, bp_alpha=1.0, bp_tol=1e-13, bp_max_sweeps=200)


def chain_error():
    N, J, h, dt, n = 5, 1.0, 0.7, 0.1, 5
    out, _ = run.simulate(dict(Lx=N, Ly=1, J=J, h=h, dt=dt, order=1, obs=(0, 0), **EXACT), nsteps=n)
    return np.max(np.abs(np.array([r["C"] for r in out]) - autocorrelation_zzx_edge(N, J, h, dt, 1, n)))


def loop_error():
    cfg = run.full_config(dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, **EXACT))
    net = pepo.Network(3, 3, cfg["obs"])
    err = 0.0
    for step in range(1, 3):
        run.trotter_step(net, cfg)
        d = dense.evolve(3, 3, 1.0, 1.0, 0.05, 1, step, cfg["obs"])
        err = max(err, np.max(np.abs(contract.to_dense(net) - d["O"])))
    return err


def star_error():
    cfg = dict(Lx=3, Ly=3, J=1.0, h=0.0, dt=0.1, order=1, obs=(1, 0), obs_pauli="X",
               chi_max=16, eps_cut=1e-12, bp_tol=1e-13, bp_max_sweeps=200)
    out, _ = run.simulate(cfg, nsteps=12)
    return np.max(np.abs(np.array([r["C"] for r in out]) - np.cos(2 * np.arange(13) * 0.1) ** 3))


def test_unpatched_oracle_passes():
    assert chain_error() < 1e-9 and loop_error() < 1e-8 and star_error() < 1e-10


def test_wrong_gate_conjugation_is_caught(monkeypatch):
    # g O g^dagger instead of g^dagger O g: breaks the dense/network agreement
    orig = pepo.bond_update

    def bad(net, v1, v2, g, *a):
        return orig(net, v1, v2, g.conj().T, *a)
    monkeypatch.setattr(pepo, "bond_update", bad)
    monkeypatch.setattr(run, "bond_update", bad)
    assert loop_error() > 1e-6


def schmidt_error():
    # gate-time lam on a chain against the dense operator-Schmidt values
    N, J, h, dt, n = 6, 1.0, 0.8, 0.1, 4
    c = run.full_config(dict(Lx=N, Ly=1, J=J, h=h, dt=dt, order=1, obs=(2, 0), **EXACT))
    want = []
    dense.evolve(N, 1, J, h, dt, 1, n, (2, 0),
                 on_bond=lambda s, v1, v2, O: want.append(dense.operator_schmidt_values(O, N, v2)))
    net = pepo.Network(N, 1, (2, 0))
    got = []
    for step in range(n):
        rec = []
        run.trotter_step(net, c, rec)
        got.extend(r["lam"] for (_, _, r) in rec)
        run.measure(net, c)
    return max(np.max(np.abs(g[:min(len(g), len(w))] - w[:min(len(g), len(w))]))
               for g, w in zip(got, want))


def test_dropped_environment_absorption_is_caught(monkeypatch):
    # identity instead of sqrt(M): the gate-time singular values are no longer
    # the operator-Schmidt values (the environment only matters for them and
    # for truncation)
    assert schmidt_error() < 1e-9
    monkeypatch.setattr(pepo, "env_sqrt", lambda M, rel: (np.eye(M.shape[0]), np.eye(M.shape[0])))
    assert schmidt_error() > 1e-6


def test_transposed_second_factor_is_caught(monkeypatch):
    # sqrt(S) V^H reshaped with the bond and Pauli indices swapped
    orig_svd = np.linalg.svd

    def bad_svd(a, full_matrices=True, compute_uv=True, **kw):
        if not compute_uv:
            return orig_svd(a, full_matrices=full_matrices, compute_uv=False, **kw)
        U, s, Vh = orig_svd(a, full_matrices=full_matrices, **kw)
        return U, s, Vh.conj()
    monkeypatch.setattr(pepo.np.linalg, "svd", bad_svd)
    assert loop_error() > 1e-6 or chain_error() > 1e-6


def test_missing_sign_tracking_is_caught(monkeypatch):
    # dropping the phase of vs_v / Z_e flips negative C(t) to positive
    orig = obp.bethe

    def bad(net, t, m, M):
        r = orig(net, t, m, M)
        r["C"] = abs(r["C"])
        return r
    monkeypatch.setattr(obp, "bethe", bad)
    monkeypatch.setattr(run, "bethe", bad)
    assert star_error() > 0.1


def test_wrong_site_gate_angle_is_caught(monkeypatch):
    # a Trotter split with the full field angle in both halves
    orig = gates.step_schedule

    def bad(gateset, J, h, dt, order):
        return orig(gateset, J, 2 * h, dt, order)
    monkeypatch.setattr(gates, "step_schedule", bad)
    monkeypatch.setattr(run.G, "step_schedule", bad)
    assert chain_error() > 1e-6


def test_dropped_pinv_of_deabsorb_is_caught(monkeypatch):
    # deabsorbing with sqrt(M) instead of M^{-1/2}
    orig = pepo.env_sqrt
    monkeypatch.setattr(pepo, "env_sqrt", lambda M, rel: (orig(M, rel)[0], orig(M, rel)[0]))
    assert chain_error() > 1e-6 or loop_error() > 1e-6


def test_dropped_first_site_gates_are_caught(monkeypatch):
    # the first layer of site gates skipped: the operator cannot leave its
    # site in the first step, so the light-cone pin must fail
    from tests import test_oracle_structure as ts
    orig = run.apply_site_gates
    calls = {"n": 0}

    def skip_first(net, g):
        calls["n"] += 1
        if calls["n"] > 1:
            orig(net, g)

    monkeypatch.setattr(run, "apply_site_gates", skip_first)
    with pytest.raises(AssertionError):
        ts.test_bond_dimension_grows_exactly_inside_the_light_cone((2, 1), 2, 1, "ZZ_X")


def chain_weights(M_of=None, pauli=None, monkeypatch=None):
    """Pauli weights of a 6-site chain after 4 untruncated steps (BP exact on
    a tree), one bond regauged by a non-orthogonal X X^-1 so that its two
    messages differ, against the dense operator's weights; M_of maps the
    converged messages to the ones handed to the weights (a planted mistake)."""
    N, nsteps = 6, 4
    cfg = run.full_config(dict(Lx=N, Ly=1, J=1.0, h=0.7, dt=0.1, order=2, obs=(2, 0), chi_max=64, eps_cut=0.0,
                               bp_alpha=1.0, bp_tol=1e-14, bp_max_sweeps=200))
    net = pepo.Network(N, 1, cfg["obs"], "Z")
    for _ in range(nsteps):
        run.trotter_step(net, cfg)
    a, b = 2, 3
    ka, kb = net.axis(a, b), net.axis(b, a)
    X = np.eye(net.O[a].shape[ka]) + 0.4 * np.random.default_rng(5).standard_normal((net.O[a].shape[ka],) * 2)
    net.O[a] = pepo.leg_apply(net.O[a], ka, X.T)
    net.O[b] = pepo.leg_apply(net.O[b], kb, np.linalg.inv(X))
    run.measure(net, cfg)
    ref = dense.site_pauli_weights(dense.evolve(N, 1, 1.0, 0.7, 0.1, 2, nsteps, (2, 0))["O"], N)
    M = net.M if M_of is None else M_of(net.M)
    if pauli is not None:
        monkeypatch.setattr(obp.G, "PAULI_BY_INDEX", pauli)
    w = obp.pauli_weights(net, M)
    return float(np.max(np.abs(w - ref)))


def test_unpatched_pauli_weights_pass():
    assert chain_weights() < 1e-10


def test_messages_of_the_wrong_direction_are_caught():
    # M_{v->u} contracted on v's leg instead of M_{u->v}
    assert chain_weights(lambda M: {(u, v): M[(v, u)] for (u, v) in M}) > 1e-3


def test_dropped_environment_is_caught():
    # the bare site tensor's weights (identity messages)
    assert chain_weights(lambda M: {k: np.eye(m.shape[0]) for k, m in M.items()}) > 1e-3


def test_swapped_pauli_components_are_caught(monkeypatch):
    # Y and Z exchanged when the weights are read off
    P = list(gates.PAULI_BY_INDEX)
    assert chain_weights(pauli=[P[0], P[1], P[3], P[2]], monkeypatch=monkeypatch) > 1e-3
