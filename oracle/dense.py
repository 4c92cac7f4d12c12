"""Brute-force dense operator evolution (test infrastructure).

The observable O(0) = P_c (a Pauli on one site) is stored as a full
2^N x 2^N complex128 matrix and every gate of the schedule is applied by
literal conjugation O -> g^dagger O g (Eq. 5).  The autocorrelation is
C(t) = Tr[O(t) P_c] / 2^N (Eq. 4) and the normalised Hilbert-Schmidt norm is
Tr[O(t)^dagger O(t)] / 2^N, which unitarity keeps at 1.

This is the definition written out; it is exact up to rounding for N <= ~10.

Pinned by: tests/test_oracle_dense.py -- C = cos(2 h t) at J = 0,
C = 1 (ZZ_X) / cos(2 J t)^deg (XX_Z) at h = 0, unit norm, and the
free-fermion (Majorana) solution of the 1 x N chain, which is an independent
method.
"""
import numpy as np

from . import gates as G
from .lattice import bonds_by_colour, site_index


def _apply_1q(O, N, q, g):
    """O -> g^dagger O g with g acting on qubit q (qubit 0 = most significant)."""
    T = O.reshape([2] * (2 * N))
    gd = g.conj().T
    # left factor acts on row index q
    T = np.tensordot(gd, T, axes=([1], [q]))
    T = np.moveaxis(T, 0, q)
    # right factor acts on column index N + q
    T = np.tensordot(T, g, axes=([N + q], [0]))
    T = np.moveaxis(T, -1, N + q)
    return T.reshape(2 ** N, 2 ** N)


def _apply_2q(O, N, q1, q2, g):
    """O -> g^dagger O g with the 4x4 unitary g acting on qubits (q1, q2)."""
    T = O.reshape([2] * (2 * N))
    g4 = g.reshape(2, 2, 2, 2)              # [out1, out2, in1, in2]
    gd4 = g.conj().T.reshape(2, 2, 2, 2)
    T = np.tensordot(gd4, T, axes=([2, 3], [q1, q2]))
    T = np.moveaxis(T, [0, 1], [q1, q2])
    T = np.tensordot(T, g4, axes=([N + q1, N + q2], [0, 1]))
    T = np.moveaxis(T, [-2, -1], [N + q1, N + q2])
    return T.reshape(2 ** N, 2 ** N)


def observable(N, site, pauli="Z"):
    mats = [G.I2] * N
    mats[site] = G.PAULI[pauli]
    out = np.array([[1.0 + 0j]])
    for m in mats:
        out = np.kron(out, m)
    return out


def evolve(Lx, Ly, J, h, dt, order, nsteps, obs_xy, gateset="ZZ_X", obs_pauli="Z",
           on_bond=None):
    """Dense Trotter evolution.  Returns dict with C[t], norm[t] for t = 0..nsteps.

    ``on_bond(step, v1, v2, O)`` is called after every bond gate (used by the
    Schmidt-value pins on chains).
    """
    N = Lx * Ly
    if N > 12:
        raise ValueError("dense evolution is limited to N <= 12")
    c = site_index(obs_xy[0], obs_xy[1], Lx)
    P = observable(N, c, obs_pauli)
    O = P.copy()
    colours = bonds_by_colour(Lx, Ly)
    sched = G.step_schedule(gateset, J, h, dt, order)
    C = [np.real(np.trace(O @ P)) / 2 ** N]
    nrm = [np.real(np.trace(O.conj().T @ O)) / 2 ** N]
    for step in range(nsteps):
        for op in sched:
            if op[0] == "site":
                for v in range(N):
                    O = _apply_1q(O, N, v, op[1])
            else:
                for (v1, v2, _, _) in colours[op[1]]:
                    O = _apply_2q(O, N, v1, v2, op[2])
                    if on_bond is not None:
                        on_bond(step, v1, v2, O)
        C.append(np.real(np.trace(O @ P)) / 2 ** N)
        nrm.append(np.real(np.trace(O.conj().T @ O)) / 2 ** N)
    return {"C": np.array(C), "norm": np.array(nrm), "O": O}


def operator_schmidt_values(O, N, cut):
    """Normalised operator-Schmidt values of O across qubits [0, cut) | [cut, N).

    O is viewed as a vector in the product of the N local operator spaces
    (each 4-dimensional: the pair (s, s')), reshaped to 4^cut x 4^(N-cut).
    """
    T = O.reshape([2] * (2 * N))
    perm = [a for q in range(N) for a in (q, N + q)]
    T = np.transpose(T, perm).reshape(4 ** cut, 4 ** (N - cut))
    s = np.linalg.svd(T, compute_uv=False)
    return s / np.linalg.norm(s)


def site_pauli_weights(O, N):
    """Pauli weights of every site of the dense operator O (Sec. 6.4 n(r, t)):
    writing O = sum_p P_p (on qubit r) (x) B_p, the weight of p at r is
    ||B_p||^2 / sum_q ||B_q||^2 (B_p = Tr_r[(P_p (x) 1) O] / 2).  Returns an
    N x 4 array (I, X, Y, Z)."""
    T = O.reshape([2] * (2 * N))
    out = np.zeros((N, 4))
    for r in range(N):
        for p, P in enumerate(G.PAULI_BY_INDEX):
            # contract P[b, a] with T[..., a (row r), ..., b (column r), ...]
            B = np.tensordot(P, T, axes=([1, 0], [r, N + r])) / 2.0
            out[r, p] = float(np.sum(np.abs(B) ** 2))
        out[r] /= np.sum(out[r])
    return out
