"""Shared helpers of the GPU tests: run the CUDA path and the oracle on one config."""
import numpy as np

import paper_2606_30985_gb300 as pkg
from oracle import run as oracle_run


def oracle_cfg(cfg):
    return dict(Lx=cfg.Lx, Ly=cfg.Ly, J=cfg.J, h=cfg.h, dt=cfg.dt, order=cfg.order,
                obs=cfg.obs, obs_pauli=cfg.obs_pauli, chi_max=cfg.chi_max, eps_cut=cfg.eps_cut,
                bp_alpha=cfg.bp_alpha, bp_tol=cfg.bp_tol, bp_max_sweeps=cfg.bp_max_sweeps,
                gateset=cfg.gateset, pinv_rel=cfg.pinv_rel)


def gpu_run(cfg, nsteps):
    eng = pkg.Engine(cfg)
    recs = eng.run(nsteps)
    lam = {b: eng.spectrum(0, b) for b in range(eng.num_bonds(0))}
    eng.close()
    return recs, lam


def oracle_bond_lams(net, Lx, Ly):
    """Oracle lam per GPU bond id (horizontal y*(Lx-1)+x, then vertical)."""
    out = {}
    for y in range(Ly):
        for x in range(Lx - 1):
            a, b = y * Lx + x, y * Lx + x + 1
            out[y * (Lx - 1) + x] = net.lam[(a, b)]
    for y in range(Ly - 1):
        for x in range(Lx):
            a, b = y * Lx + x, (y + 1) * Lx + x
            out[Ly * (Lx - 1) + y * Lx + x] = net.lam[(a, b)]
    return out


# floor of the per-value relative check of the spectra: values below it carry
# little weight and their relative error is set by the absolute one
LAM_REL_FLOOR = 1e-2


def lam_errors(lam, lref):
    """(max |l_k - r_k| over bonds with lam_0 = 1 normalisation and the
    unmatched tail, max |l_k - r_k| / r_k over r_k >= LAM_REL_FLOOR r_0)."""
    lam_err, rel_err = 0.0, 0.0
    for b, l in lam.items():
        r = lref[b]
        k = min(len(l), len(r))
        e = np.max(np.abs(l[:k] - r[:k])) if k else 0.0
        tail = max(np.max(l[k:], initial=0.0), np.max(r[k:], initial=0.0))
        lam_err = max(lam_err, e, tail)
        if k:
            sel = r[:k] >= LAM_REL_FLOOR * r[0]
            rel_err = max(rel_err, float(np.max(np.abs(l[:k][sel] - r[:k][sel]) / r[:k][sel])))
    return lam_err, rel_err


def compare(cfg, nsteps):
    recs, lam = gpu_run(cfg, nsteps)
    ref, net = oracle_run.simulate(oracle_cfg(cfg), nsteps=nsteps)
    C = np.array([r["C"] for r in recs])
    Cr = np.array([r["C"] for r in ref])
    lref = oracle_bond_lams(net, cfg.Lx, cfg.Ly)
    lam_err, lam_rel = lam_errors(lam, lref)
    # the Q-less update equals the literal one only with full-rank messages
    # (flags bit 0 marks a rank-deficient one): a parity pass must not hide it
    flags = 0
    for r in recs:
        flags |= int(r["flags"])
    return dict(C=C, Cref=Cr, dC=float(np.max(np.abs(C - Cr))), lam_err=lam_err, lam_rel=lam_rel,
                flags=flags, recs=recs, ref=ref)
