"""Free-fermion (Majorana) solution of the Trotterised 1 x N Ising chain.

An independent method used only to pin the oracle.  Jordan-Wigner:
  g_{2j} = (prod_{k<j} Z_k) X_j,   g_{2j+1} = (prod_{k<j} Z_k) Y_j,
so Z_j = -i g_{2j} g_{2j+1} and X_j X_{j+1} = -i g_{2j+1} g_{2j+2}.  A gate
exp(-i theta (-i g_a g_b)) conjugates the Majoranas by a plane rotation:
  g_a -> cos(2 theta) g_a - sin(2 theta) g_b,  g_b -> cos(2 theta) g_b + sin(2 theta) g_a,
so a whole gate sequence is one real orthogonal 2N x 2N matrix R (product of
the rotations in application order).  At infinite temperature
  Tr[Z_j(t) Z_j] / 2^N = R[2j,2j] R[2j+1,2j+1] - R[2j,2j+1] R[2j+1,2j]
(XX bonds, Z field), and for ZZ bonds with an X field a global Hadamard maps
Z_0 to X_0 = g_0, giving Tr[Z_0(t) Z_0] / 2^N = R[0, 0].
"""
import numpy as np


def _rot(n2, a, b, theta):
    r = np.eye(n2)
    c, s = np.cos(2 * theta), np.sin(2 * theta)
    r[a, a] = c
    r[a, b] = -s
    r[b, a] = s
    r[b, b] = c
    return r


def majorana_rotation(N, J, h, dt, order, nsteps):
    """R after each step for XX bonds (angle J dt) and Z sites (h dt or h dt / 2)."""
    n2 = 2 * N
    phi = h * dt if order == 1 else 0.5 * h * dt
    site = np.eye(n2)
    for j in range(N):
        site = site @ _rot(n2, 2 * j, 2 * j + 1, phi)
    bonds = np.eye(n2)
    for parity in (0, 1):                      # colour 0: even x, colour 1: odd x
        for j in range(parity, N - 1, 2):
            bonds = bonds @ _rot(n2, 2 * j + 1, 2 * j + 2, J * dt)
    step = site @ bonds @ site if order == 2 else site @ bonds
    out = [np.eye(n2)]
    R = np.eye(n2)
    for _ in range(nsteps):
        R = R @ step
        out.append(R.copy())
    return out


def autocorrelation_xxz(N, j, J, h, dt, order, nsteps):
    Rs = majorana_rotation(N, J, h, dt, order, nsteps)
    a, b = 2 * j, 2 * j + 1
    return np.array([R[a, a] * R[b, b] - R[a, b] * R[b, a] for R in Rs])


def autocorrelation_zzx_edge(N, J, h, dt, order, nsteps):
    Rs = majorana_rotation(N, J, h, dt, order, nsteps)
    return np.array([R[0, 0] for R in Rs])
