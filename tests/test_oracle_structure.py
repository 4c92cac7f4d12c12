"""Structural pins of the oracle: the gate tables, the discrete light cone of
the Trotter schedule, and the C4 symmetry of the converged BP environments.

Expected values come from the mathematics, not from the oracle:
* g = exp(-i phi X) acting on Z gives g^dagger Z g = cos(2 phi) Z + sin(2 phi) Y
  (worked by hand from XZ = -iY, ZX = iY, XZX = -Z); Pauli transfer matrices
  of unitaries are real orthogonal, and the identity at angle 0.
* Light cone.  A bond gate exp(-i a P(x)P) leaves a site operator in span{I, P}
  alone; acting on a site whose operator has parts outside span{I, P} (an
  "active" site), it puts only I and P on the other site.  So a site reached
  through a bond is inactive until the next layer of site gates (rotations
  about the other Pauli) activates every site of the support.  Propagating
  that rule through the stated schedule (site gates, then colours 0..3 =
  horizontal even x, horizontal odd x, vertical even y, vertical odd y;
  rebuilt here, not taken from the oracle) predicts exactly which bonds a
  gate hits with an active end: those and only those get chi > 1; every
  other bond keeps chi = 1 and lambda = 1.  ("No truncation" below is a
  relative cut of 1e-12: a cut of 0 would keep the exactly-zero singular
  values of a trivial bond as bond dimension.)
* With ZZ bond gates every bond gate of a step commutes with the others, so
  the step is C4-symmetric on an odd grid with the observable at the centre
  whatever the colour order.  Without truncation the network is the exact
  evolved operator, and the eigenvalues of M_ab M_ba^T (normalised) are
  invariant under a change of gauge on the bond: they must agree on bonds
  that a 90-degree rotation maps onto each other.
"""
import math

import numpy as np
import pytest

from oracle import gates as G
from oracle.bp import bp_double
from oracle.pepo import bond_key
from oracle.run import simulate

PAULIS = [G.I2, G.X2, G.Y2, G.Z2]


def ptm(U):
    """Pauli transfer matrix R[a, b] = Tr(P_a U^dagger P_b U) / 2^q."""
    q = int(round(math.log2(U.shape[0])))
    basis = PAULIS if q == 1 else [np.kron(a, b) for a in PAULIS for b in PAULIS]
    d = U.shape[0]
    R = np.array([[np.trace(Pa @ U.conj().T @ Pb @ U) / d for Pb in basis] for Pa in basis])
    assert np.max(np.abs(R.imag)) < 1e-14
    return R.real


@pytest.mark.parametrize("gateset", ["ZZ_X", "XX_Z"])
def test_gate_transfer_matrices_are_orthogonal_and_identity_at_zero(gateset):
    for theta in (0.0, 0.05, 0.37, 1.1):
        for U in (G.site_unitary(gateset, theta), G.bond_unitary(gateset, theta)):
            R = ptm(U)
            assert np.max(np.abs(R.T @ R - np.eye(len(R)))) < 1e-14
            if theta == 0.0:
                assert np.max(np.abs(R - np.eye(len(R)))) < 1e-15


def test_site_gate_rotates_z_into_y():
    for phi in (0.05, 0.3, 1.2):
        g = G.site_unitary("ZZ_X", phi)
        out = g.conj().T @ G.Z2 @ g
        want = math.cos(2 * phi) * G.Z2 + math.sin(2 * phi) * G.Y2
        assert np.max(np.abs(out - want)) < 1e-15


def _colours(Lx, Ly):
    """Bonds of each colour, from the schedule's definition (independent of the
    oracle's lattice module)."""
    col = {0: [], 1: [], 2: [], 3: []}
    for y in range(Ly):
        for x in range(Lx - 1):
            col[0 if x % 2 == 0 else 1].append((y * Lx + x, y * Lx + x + 1))
    for y in range(Ly - 1):
        for x in range(Lx):
            col[2 if y % 2 == 0 else 3].append((y * Lx + x, (y + 1) * Lx + x))
    return col


def light_cone(Lx, Ly, obs, steps, order):
    """Bonds that a gate hits with an active end (rule in the module docstring)."""
    col = _colours(Lx, Ly)
    support = {obs[1] * Lx + obs[0]}
    active = set()
    hit = set()
    for _ in range(steps):
        active = set(support)                      # site gates (h dt, or h dt / 2)
        for c in range(4):
            for (u, v) in col[c]:
                if u in active or v in active:
                    hit.add(bond_key(u, v))
                    support |= {u, v}              # the other end joins, inactive
        if order == 2:
            active = set(support)                  # closing half site gates
    return hit, col


@pytest.mark.parametrize("gateset", ["ZZ_X", "XX_Z"])
@pytest.mark.parametrize("obs,steps,order", [((0, 0), 2, 1), ((2, 1), 2, 1), ((1, 2), 3, 2), ((4, 3), 2, 2)])
def test_bond_dimension_grows_exactly_inside_the_light_cone(obs, steps, order, gateset):
    Lx, Ly = 5, 4
    cfg = dict(Lx=Lx, Ly=Ly, J=0.9, h=1.3, dt=0.2, order=order, obs=obs, chi_max=64, eps_cut=1e-12,
               bp_max_sweeps=3, gateset=gateset, obs_pauli="Z" if gateset == "ZZ_X" else "X")
    _, net = simulate(cfg, nsteps=steps)
    hit, col = light_cone(Lx, Ly, obs, steps, order)
    grown = set()
    for (u, v) in [b for c in range(4) for b in col[c]]:
        k = bond_key(u, v)
        if net.chi(u, v) > 1:
            grown.add(k)
        else:
            assert np.array_equal(net.lam[k], [1.0]), (k, net.lam[k])
    assert grown == hit, (sorted(grown ^ hit))
    assert 0 < len(hit) < sum(len(col[c]) for c in range(4))


def _rot90(v, L):
    x, y = v % L, v // L
    return x * L + (L - 1 - y)   # (x, y) -> (L - 1 - y, x)


def test_converged_environments_are_c4_symmetric():
    L = 3
    cfg = dict(Lx=L, Ly=L, J=1.0, h=1.7, dt=0.15, order=2, obs=(1, 1), chi_max=256, eps_cut=1e-12,
               gateset="ZZ_X", bp_max_sweeps=3)
    _, net = simulate(cfg, nsteps=2)
    sweeps, delta = bp_double(net, 0.5, 1e-13, 4000)
    assert delta < 1e-12
    spec = {}
    for (a, b) in net.M:
        if a < b:
            P = net.M[(a, b)] @ net.M[(b, a)].T
            w = np.sort(np.abs(np.linalg.eigvals(P)))[::-1]
            spec[(a, b)] = w / w.sum()
    assert max(len(w) for w in spec.values()) > 1       # the bonds are entangled
    for (a, b), w in spec.items():
        ra, rb = _rot90(a, L), _rot90(b, L)
        w2 = spec[(min(ra, rb), max(ra, rb))]
        assert len(w) == len(w2)
        assert np.max(np.abs(w - w2)) < 1e-10, ((a, b), w, w2)
