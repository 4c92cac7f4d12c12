"""Seeded synthetic saturated states (every bond at chi_max).

Shapes follow the library's conventions: site tensors in the canonical layout
(legs U, D, L, R that exist, then the Pauli index I, X, Y, Z); bonds numbered
horizontal first (y * (Lx - 1) + x) then vertical (Ly * (Lx - 1) + y * Lx + x).
Values: Gaussian entries, each bond leg weighted by sqrt(lam) with a
geometrically decaying lam (the shape of a saturated Schmidt spectrum), the
identity Pauli component weighted up; messages diag(lam) on both directions.
"""
import numpy as np


def bond_list(Lx, Ly):
    bonds = []
    for y in range(Ly):
        for x in range(Lx - 1):
            bonds.append((y * Lx + x, y * Lx + x + 1))
    for y in range(Ly - 1):
        for x in range(Lx):
            bonds.append((y * Lx + x, (y + 1) * Lx + x))
    return bonds


def site_legs(Lx, Ly, v):
    """(neighbour, bond id) of each present leg of site v in canonical order U, D, L, R."""
    x, y = v % Lx, v // Lx
    legs = []
    if y > 0:
        legs.append(((y - 1) * Lx + x, Ly * (Lx - 1) + (y - 1) * Lx + x))
    if y < Ly - 1:
        legs.append(((y + 1) * Lx + x, Ly * (Lx - 1) + y * Lx + x))
    if x > 0:
        legs.append((y * Lx + x - 1, y * (Lx - 1) + x - 1))
    if x < Lx - 1:
        legs.append((y * Lx + x + 1, y * (Lx - 1) + x))
    return legs


def saturated_state(Lx, Ly, chi, seed=0, decay=0.06, dtype=np.float64):
    rng = np.random.default_rng(seed)
    nb = len(bond_list(Lx, Ly))
    lam = np.exp(-decay * np.arange(chi))
    lam = lam / np.linalg.norm(lam)
    lams = np.zeros((nb, chi))
    lams[:] = lam
    sq = np.sqrt(lam)
    pw = np.array([1.0, 0.5, 0.5, 0.5])
    sites = []
    for v in range(Lx * Ly):
        legs = site_legs(Lx, Ly, v)
        shape = tuple([chi] * len(legs)) + (4,)
        t = rng.standard_normal(shape).astype(dtype)
        for k in range(len(legs)):
            sh = [1] * (len(legs) + 1)
            sh[k] = chi
            t *= sq.reshape(sh).astype(dtype)
        t *= pw.astype(dtype)
        t /= np.sqrt(np.mean(t.astype(np.float64) ** 2)) * np.sqrt(t.size) ** (1.0 / 3.0)
        sites.append(t)
    msgs = np.zeros((nb, 2, chi, chi))
    for b in range(nb):
        msgs[b, 0] = np.diag(lam)
        msgs[b, 1] = np.diag(lam)
    chis = np.full(nb, chi, dtype=np.int32)
    return dict(sites=sites, chi=chis, lam=lams, msgs=msgs)
