"""Seeded synthetic saturated states (every bond at chi_max).

Shapes follow the library's conventions: site tensors in the canonical layout
(legs U, D, L, R that exist, then the Pauli index I, X, Y, Z); bonds numbered
horizontal first (y * (Lx - 1) + x) then vertical (Ly * (Lx - 1) + y * Lx + x).
Values: Gaussian entries, each bond leg weighted by sqrt(lam) with a
geometrically decaying lam (the shape of a saturated Schmidt spectrum), the
identity Pauli component weighted up; messages diag(lam) on both directions.
The Pauli component that the correlator's single-layer network pins (the
identity, and Z at the observable site) is drawn half-normal (|Gaussian|)
instead of Gaussian: the pinned network is then positive and single-layer
vector BP converges (Perron-Frobenius), as it does on evolved operators;
with signed Gaussian slices it does not (residual ~1.4 after 100 sweeps on
6x6, chi = 10).  The other three components stay Gaussian, so every bond
keeps a full decaying spectrum at chi_max.
Every site has its own seed (seed, site), so one site can be regenerated
without the others.
"""
import numpy as np

DECAY = 0.06
PAULI_WEIGHT = np.array([1.0, 0.5, 0.5, 0.5])


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


def spectrum(chi, decay=DECAY):
    lam = np.exp(-decay * np.arange(chi))
    return lam / np.linalg.norm(lam)


def site_tensor(Lx, Ly, chi, seed, v, dtype=np.float64, decay=DECAY, obs=None):
    """obs: (x, y) of the observable site, whose pinned component is Z (index 3)."""
    legs = site_legs(Lx, Ly, v)
    rng = np.random.default_rng([seed, v])
    shape = tuple([chi] * len(legs)) + (4,)
    t = rng.standard_normal(shape, dtype=np.float32 if dtype == np.float32 else np.float64)
    pin = 3 if (obs is not None and v == obs[1] * Lx + obs[0]) else 0
    np.abs(t[..., pin], out=t[..., pin])
    sq = np.sqrt(spectrum(chi, decay)).astype(t.dtype)
    for k in range(len(legs)):
        sh = [1] * (len(legs) + 1)
        sh[k] = chi
        t *= sq.reshape(sh)
    t *= PAULI_WEIGHT.astype(t.dtype)
    return t


def bond_data(Lx, Ly, chi, decay=DECAY):
    nb = len(bond_list(Lx, Ly))
    lam = spectrum(chi, decay)
    lams = np.tile(lam, (nb, 1))
    msgs = np.zeros((nb, 2, chi, chi))
    msgs[:, 0] = np.diag(lam)
    msgs[:, 1] = np.diag(lam)
    return dict(chi=np.full(nb, chi, dtype=np.int32), lam=lams, msgs=msgs)


def saturated_state(Lx, Ly, chi, seed=0, dtype=np.float64, decay=DECAY, obs=None):
    st = bond_data(Lx, Ly, chi, decay)
    st["sites"] = [site_tensor(Lx, Ly, chi, seed, v, dtype, decay, obs) for v in range(Lx * Ly)]
    return st
