"""GPU path (through the C ABI) against the CPU oracle and closed forms.

Tolerances: FP64 path |dC| <= 1e-8 and lam error (relative to lam_0) <= 1e-6;
FP32 path |dC| <= 1e-5 (the FP32-path bound of the parity target) and lam
error <= 1e-5.  The per-value relative error of the spectra, over values at
least 1e-2 of lam_0, is held to 100 times that bound (the absolute bound at
the floor).  Every oracle comparison also asserts flags bit 0 clear: with a
rank-deficient message the GPU's Q-less update departs from the literal
projector of the oracle.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from tests.free_fermion import autocorrelation_zzx_edge
from tests.gpu_common import compare, gpu_run

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-8, 1e-6), "fp32": (1e-5, 1e-5)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_J0_closed_form(prec):
    cfg = pkg.Config(Lx=3, Ly=3, J=0.0, h=1.1, dt=0.05, chi_max=4, precision=prec, bp_tol=1e-10)
    recs, _ = gpu_run(cfg, 10)
    C = np.array([r["C"] for r in recs])
    ref = np.cos(2 * 1.1 * 0.05 * np.arange(11))
    assert np.max(np.abs(C - ref)) < TOL[prec][0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_h0_closed_form(prec):
    cfg = pkg.Config(Lx=3, Ly=3, J=1.0, h=0.0, dt=0.05, chi_max=4, precision=prec, bp_tol=1e-10)
    recs, _ = gpu_run(cfg, 8)
    assert max(abs(r["C"] - 1.0) for r in recs) < TOL[prec][0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_star_tree_sign_tracking(prec):
    cfg = pkg.Config(Lx=3, Ly=3, J=1.0, h=0.0, dt=0.1, obs=(1, 0), obs_pauli="X", chi_max=16,
                     precision=prec, bp_tol=1e-12 if prec == "fp64" else 1e-7, eps_cut=1e-12)
    recs, _ = gpu_run(cfg, 12)
    C = np.array([r["C"] for r in recs])
    ref = np.cos(2 * np.arange(13) * 0.1) ** 3
    assert ref.min() < -0.1
    assert np.max(np.abs(C - ref)) < TOL[prec][0]


def test_chain_is_exact_free_fermions():
    N, J, h, dt, n = 6, 1.0, 0.7, 0.1, 8
    cfg = pkg.Config(Lx=N, Ly=1, J=J, h=h, dt=dt, obs=(0, 0), chi_max=64, eps_cut=1e-13,
                     bp_alpha=1.0, bp_tol=1e-13, bp_max_sweeps=200, precision="fp64")
    recs, _ = gpu_run(cfg, n)
    C = np.array([r["C"] for r in recs])
    assert np.max(np.abs(C - autocorrelation_zzx_edge(N, J, h, dt, 1, n))) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_3x3_chi8_parity(prec):
    cfg = pkg.Config(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=8, bp_alpha=0.5,
                     bp_tol=1e-10 if prec == "fp64" else 1e-7, precision=prec)
    r = compare(cfg, 20)
    assert r["dC"] < TOL[prec][0], r["dC"]
    assert r["lam_err"] < TOL[prec][1], r["lam_err"]
    assert r["lam_rel"] < 100 * TOL[prec][1], r["lam_rel"]
    assert r["flags"] & 1 == 0


def test_config2_4x4_offcentre_fp32_parity():
    cfg = pkg.Config(Lx=4, Ly=4, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=20,
                     precision="fp32")
    r = compare(cfg, 10)
    assert r["dC"] < 1e-5, r["dC"]
    assert r["lam_err"] < 1e-5, r["lam_err"]
    assert r["lam_rel"] < 1e-3, r["lam_rel"]
    assert r["flags"] & 1 == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_qr_branch_independence(prec):
    # Householder-only vs Cholesky-QR-only: the R-factors differ by an orthogonal
    # factor, so C and lam must agree (Sec. 4.2: both are QR factorisations).
    base = dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=8, precision=prec, bp_tol=1e-9)
    hh, lh = gpu_run(pkg.Config(qr_n_thresh=10 ** 9, **base), 12)
    ch, lc = gpu_run(pkg.Config(qr_n_thresh=0, qr_ratio_thresh=0.0, **base), 12)
    tol = TOL[prec][0]
    assert max(abs(a["C"] - b["C"]) for a, b in zip(hh, ch)) < tol
    for b in lh:
        k = min(len(lh[b]), len(lc[b]))
        assert np.max(np.abs(lh[b][:k] - lc[b][:k])) < TOL[prec][1]


@pytest.mark.parametrize("cfgname", ["c1", "c2"])
def test_tf32x3_mixed_precision_parity(cfgname):
    # Mixed-precision path: Gram / absorb / BP contractions on the tensor cores
    # with the three-product TF32 split; bound |dC| <= 1e-3 (mixed-precision
    # target), lam error <= 1e-4.
    if cfgname == "c1":
        cfg = pkg.Config(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=8, bp_tol=1e-7,
                         precision="tf32x3")
        n = 20
    else:
        cfg = pkg.Config(Lx=4, Ly=4, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=20,
                         precision="tf32x3")
        n = 8
    r = compare(cfg, n)
    assert r["dC"] < 1e-3, r["dC"]
    assert r["lam_err"] < 1e-4, r["lam_err"]
    assert r["lam_rel"] < 1e-2, r["lam_rel"]
    assert r["flags"] & 1 == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_colour_calls_equal_one_step(prec):
    # pepo_trotter_colour 0..3 is exactly pepo_trotter_step: same launches in
    # the same order (direct instead of a graph), so bit-identical sites
    base = dict(Lx=4, Ly=3, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=12, precision=prec)
    a = pkg.Engine(pkg.Config(**base))
    b = pkg.Engine(pkg.Config(**base))
    try:
        a.trotter_step(3)
        b.trotter_step(2)
        b.trotter_colour(0)
        with pytest.raises(pkg.PepoError, match="partly applied"):
            b.bp_converge()
        with pytest.raises(pkg.PepoError, match="out of order"):
            b.trotter_colour(2)
        for col in (1, 2, 3):
            b.trotter_colour(col)
        for v in range(12):
            assert np.array_equal(a.site(0, v)[0], b.site(0, v)[0]), v
        for bond in range(a.num_bonds()):
            assert np.array_equal(a.spectrum(0, bond), b.spectrum(0, bond))
        b.bp_converge()
        a.bp_converge()
        Ca, Da = a.correlator()
        Cb, Db = b.correlator()
        assert abs(Ca[0] - Cb[0]) < 1e-12 and Da[0]["steps"] == Db[0]["steps"] == 3
    finally:
        a.close()
        b.close()
