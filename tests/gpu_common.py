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


def compare(cfg, nsteps):
    recs, lam = gpu_run(cfg, nsteps)
    ref, net = oracle_run.simulate(oracle_cfg(cfg), nsteps=nsteps)
    C = np.array([r["C"] for r in recs])
    Cr = np.array([r["C"] for r in ref])
    lref = oracle_bond_lams(net, cfg.Lx, cfg.Ly)
    lam_err = 0.0
    for b, l in lam.items():
        r = lref[b]
        k = min(len(l), len(r))
        e = np.max(np.abs(l[:k] - r[:k])) if k else 0.0
        tail = max(np.max(l[k:], initial=0.0), np.max(r[k:], initial=0.0))
        lam_err = max(lam_err, e, tail)
    return dict(C=C, Cref=Cr, dC=float(np.max(np.abs(C - Cr))), lam_err=lam_err,
                recs=recs, ref=ref)
