"""Batched instances and CUDA-graph execution.

Several independent instances of uneven size in one context run as grouped
launches (every instance's items of a wave in one launch) and, with timing
off, as replayed CUDA graphs of one Trotter step / one BP sweep / one
single-layer sweep.  Each instance must give exactly what it gives alone, and
the graph path exactly what the direct launches give, and every instance of
a batched context (the three uneven ones below, and a seeded subset of the
64-instance workload) must match the oracle run on its own configuration
(FP32 bounds: |dC| <= 1e-5, lam within 1e-5 of lam_0, flags bit 0 clear).
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import run as oracle_run
from tests.gpu_common import lam_errors, oracle_bond_lams, oracle_cfg

pytestmark = pytest.mark.gpu

CFGS = [
    dict(Lx=4, Ly=4, J=1.0, h=1.0, dt=0.05, order=2, obs=(1, 1), chi_max=8),
    dict(Lx=3, Ly=3, J=1.0, h=2.0, dt=0.05, order=1, obs=(1, 1), chi_max=6),
    dict(Lx=5, Ly=4, J=1.0, h=1.5, dt=0.05, order=2, obs=(2, 1), chi_max=10),
]


def _trajectory(eng, steps, timing=False):
    eng.set_timing(timing)
    out = []
    for _ in range(steps):
        eng.trotter_step(1)
        sw, de = eng.bp_converge()
        C, D = eng.correlator()
        out.append((list(C), list(sw)))
    return out


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_batched_instances_match_single_runs(precision):
    cfgs = [pkg.Config(precision=precision, **c) for c in CFGS]
    eng = pkg.Engine(cfgs)
    batched = _trajectory(eng, 6)
    eng.close()
    for i, cfg in enumerate(cfgs):
        e1 = pkg.Engine(cfg)
        single = _trajectory(e1, 6)
        e1.close()
        for s in range(6):
            assert batched[s][0][i] == single[s][0][0], (i, s, batched[s][0][i], single[s][0][0])
            assert batched[s][1][i] == single[s][1][0]


def test_graph_replay_matches_direct_launches():
    cfg = pkg.Config(precision="fp32", **CFGS[2])
    a = pkg.Engine(cfg)
    ga = _trajectory(a, 5, timing=False)     # graphs
    la = a.launches()
    a.close()
    b = pkg.Engine(cfg)
    gb = _trajectory(b, 5, timing=True)      # direct launches (timing on)
    lb = b.launches()
    b.close()
    assert ga == gb
    assert la == lb                          # graph replays are counted launch by launch


def test_state_snapshot_restores_the_trajectory():
    import torch
    cfg = pkg.Config(precision="tf32x3", **CFGS[0])
    eng = pkg.Engine(cfg)
    eng.trotter_step(3)
    eng.bp_converge()
    snap = torch.empty(eng.state_bytes(), dtype=torch.uint8, device="cuda")
    eng.save_state(snap)
    first = _trajectory(eng, 3)
    eng.load_state(snap)
    again = _trajectory(eng, 3)
    eng.close()
    assert first == again


def _batched_vs_oracle(cfgs, nsteps):
    eng = pkg.Engine(cfgs)
    try:
        recs = eng.run(nsteps)
        lam = [{b: eng.spectrum(i, b) for b in range(eng.num_bonds(i))} for i in range(len(cfgs))]
    finally:
        eng.close()
    worst = 0.0
    for i, cfg in enumerate(cfgs):
        ref, net = oracle_run.simulate(oracle_cfg(cfg), nsteps=nsteps)
        C = np.array([r[i]["C"] for r in recs])
        Cr = np.array([r["C"] for r in ref])
        dC = float(np.max(np.abs(C - Cr)))
        lam_err, _ = lam_errors(lam[i], oracle_bond_lams(net, cfg.Lx, cfg.Ly))
        flags = 0
        for r in recs:
            flags |= int(r[i]["flags"])
        assert dC < 1e-5, (i, dC)
        assert lam_err < 1e-5, (i, lam_err)
        assert flags & 1 == 0, i
        worst = max(worst, dC)
    return worst


def test_batched_instances_match_the_oracle():
    cfgs = [pkg.Config(precision="fp32", **c) for c in CFGS]
    _batched_vs_oracle(cfgs, 6)


def test_batched_workload_subset_matches_the_oracle():
    # the first six instances of the seeded 64-instance workload (grids 4x4
    # to 6x6, chi_max 16 / 32 / 48, h ~ U[0.5, 3]), four steps
    from workloads.configs import c3_instances
    insts = c3_instances(seed=0)[:6]
    cfgs = [pkg.Config(**{k: v for k, v in c.items() if k not in ("nsteps", "precision")}, precision="fp32")
            for c in insts]
    _batched_vs_oracle(cfgs, 4)


def test_host_checkpoint_restarts_a_fresh_context(tmp_path):
    cfg = pkg.Config(precision="tf32x3", **CFGS[0])
    a = pkg.Engine(cfg)
    try:
        a.trotter_step(3)
        a.bp_converge()
        path = str(tmp_path / "state.npz")
        assert a.checkpoint(path) == 3
        first = _trajectory(a, 2)
        _, Da = a.correlator()
    finally:
        a.close()
    b = pkg.Engine(cfg)
    try:
        assert b.restore(path) == 3
        again = _trajectory(b, 2)
        _, Db = b.correlator()
    finally:
        b.close()
    assert first == again
    assert Da[0]["steps"] == Db[0]["steps"] == 5
    other = pkg.Engine(pkg.Config(precision="tf32x3", **CFGS[1]))
    try:
        with pytest.raises(pkg.PepoError, match="another configuration"):
            other.restore(path)
    finally:
        other.close()
