"""Exact contraction of small operator networks (oracle).

Sec. 2.6 step 1: by Pauli orthogonality the trace Tr[O P]/2^N is the full
contraction of the network with every physical pair pinned (P_c at the
observable site, I elsewhere).  ``pinned_value`` does that contraction
exactly (no Bethe factorisation) and ``to_dense`` contracts the network with
the physical pairs left open, giving the 2^N x 2^N operator itself.

Only for small networks (N <= 9 and modest bond dimensions).

Pinned by: tests/test_oracle_pepo.py (the initial network contracts to P_c;
after evolution without truncation it contracts to the dense operator).
"""
import string

import numpy as np

from . import gates as G
from .pepo import bond_key

_LETTERS = string.ascii_letters


def _bond_letters(net):
    letters, i = {}, 0
    for v in range(net.N):
        for (_, u) in net.legs[v]:
            b = bond_key(u, v)
            if b not in letters:
                letters[b] = _LETTERS[i]
                i += 1
    return letters, i


def to_dense(net):
    """Contract site by site in index order, keeping the physical pairs open."""
    letters, i0 = _bond_letters(net)
    phys_s = [_LETTERS[i0 + v] for v in range(net.N)]
    phys_t = [_LETTERS[i0 + net.N + v] for v in range(net.N)]
    T, cur = None, ""
    for v in range(net.N):
        idx = "".join(letters[bond_key(u, v)] for (_, u) in net.legs[v]) + phys_s[v] + phys_t[v]
        if T is None:
            T, cur = net.O[v], idx
            continue
        shared = set(cur) & set(idx)
        out = "".join(ch for ch in cur if ch not in shared) + "".join(ch for ch in idx if ch not in shared)
        T = np.einsum(cur + "," + idx + "->" + out, T, net.O[v], optimize=True)
        cur = out
    final = "".join(phys_s) + "".join(phys_t)
    T = np.einsum(cur + "->" + final, T)
    return T.reshape(2 ** net.N, 2 ** net.N)


def pinned_value(net):
    letters, _ = _bond_letters(net)
    terms, ops = [], []
    for v in range(net.N):
        P = G.PAULI[net.obs_pauli] if v == net.obs_site else G.I2
        ops.append(np.einsum("...ab,ba->...", net.O[v], P) / 2.0)
        terms.append("".join(letters[bond_key(u, v)] for (_, u) in net.legs[v]))
    expr = ",".join(terms) + "->"
    return complex(np.einsum(expr, *ops, optimize="greedy"))
