"""Batched instances and CUDA-graph execution.

Several independent instances of uneven size in one context run as grouped
launches (every instance's items of a wave in one launch) and, with timing
off, as replayed CUDA graphs of one Trotter step / one BP sweep / one
single-layer sweep.  Each instance must give exactly what it gives alone, and
the graph path exactly what the direct launches give.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg

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
