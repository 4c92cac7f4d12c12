"""Parity at the full 10x10, chi_max = 100 size on sampled outputs.

The 10x10, chi_max = 100 FP32 workload of bench.py is started from its seeded
synthetic saturated state and advanced one Trotter step on the GPU.  The
colour-0 bonds are updated first, from the initial state alone, so the oracle
can recompute any of them one by one: for the five colour-0 bonds of the top
row (corner-edge, edge-edge and edge-corner pairs) it converts the two site
tensors, applies the half-angle site gates that the GPU folds into these bond
gates (second-order split), and performs the literal bond update with the
synthetic environment messages.  The Vidal-normalised singular values must
agree within the FP32-path bound (relative to lam_0); the TF32x3 path (leg
contractions of the absorb step on the tensor cores) within its own bound.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import gates as og
from oracle import pepo as opepo

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("tf32x3", 1e-4)])
def test_first_colour_bonds_match_oracle_at_chi100(precision, tol):
    import bench
    from workloads.synthetic import bond_data, site_tensor

    w = dict(bench.WORKLOAD)
    w["precision"] = precision
    Lx, Ly, chi = w["Lx"], w["Ly"], w["chi_max"]
    cfg = pkg.Config(**w)
    eng = pkg.Engine(cfg)
    bench.upload_state(eng, w, bench.SEED)
    eng.trotter_step(1)
    sampled = [0, 2, 4, 6, 8]                 # horizontal bonds (x, 0)-(x+1, 0), x even
    got = {b: eng.spectrum(0, b) for b in sampled}
    eng.close()

    bd = bond_data(Lx, Ly, chi)
    g2 = og.bond_unitary("ZZ_X", w["J"] * w["dt"])
    g1 = og.site_unitary("ZZ_X", 0.5 * w["h"] * w["dt"])
    for b in sampled:
        v1, v2 = b, b + 1
        sites = {v: site_tensor(Lx, Ly, chi, bench.SEED, v, np.float32, obs=w["obs"]).astype(np.float64)
                 for v in (v1, v2)}
        net = opepo.from_pauli(Lx, Ly, w["obs"], "Z", sites, bd["chi"], bd["msgs"],
                               sites_subset={v1, v2})
        opepo.apply_site_gate(net, v1, g1)
        opepo.apply_site_gate(net, v2, g1)
        r = opepo.bond_update(net, v1, v2, g2, chi, w.get("eps_cut", 1e-11), 1e-12)
        ref = r["lam"]
        gpu = got[b]
        assert len(gpu) == len(ref) == chi
        err = np.max(np.abs(gpu - ref)) / ref[0]
        assert err < tol, (b, err)
