"""Host-side parts of bench.py that need no GPU: the staged state upload
(every site reaches the engine with the generated values, through the
staging array when there is one) and the maximum site size it stages."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads.synthetic import site_tensor  # noqa: E402


class FakeEngine:
    """Records what the upload hands to the library (copies: a staging
    array is reused between calls)."""

    def __init__(self):
        self.sites = {}
        self.ptrs = set()
        self.bonds = None

    def set_bonds(self, inst, chi, lam, msgs):
        self.bonds = (np.array(chi), np.array(lam), np.array(msgs))

    def set_site(self, inst, v, t):
        self.ptrs.add(t.__array_interface__["data"][0])
        self.sites[v] = np.array(t, copy=True)


@pytest.mark.parametrize("staged", [False, True])
@pytest.mark.parametrize("grid", [(4, 3), (2, 5)])
def test_upload_sends_every_generated_site(monkeypatch, staged, grid):
    Lx, Ly = grid
    chi = 3
    w = dict(bench.WORKLOAD, Lx=Lx, Ly=Ly, chi_max=chi, obs=(1, 1))
    sizes = []

    def fake_pinned(n):
        sizes.append(n)
        return np.empty(n, dtype=np.float32) if staged else None

    monkeypatch.setattr(bench, "pinned_buffer", fake_pinned)
    eng = FakeEngine()
    total, h2d_s, pinned = bench.upload_state(eng, w, seed=7)
    assert pinned == staged and h2d_s >= 0.0
    max_deg = (Lx > 1) + (Lx > 2) + (Ly > 1) + (Ly > 2)
    assert sizes == [4 * chi ** max_deg]
    assert sorted(eng.sites) == list(range(Lx * Ly))
    nbytes = 0
    for v in range(Lx * Ly):
        ref = site_tensor(Lx, Ly, chi, 7, v, np.float32, obs=w["obs"])
        assert eng.sites[v].shape == ref.shape and np.array_equal(eng.sites[v], ref)
        nbytes += ref.nbytes
    assert total == nbytes
    if staged:
        assert len(eng.ptrs) == 1       # one staging array, reused for every site
