"""Unitaries and the Trotter schedule used by the oracle.

Model (Sec. 2.1, Eq. 1): a transverse-field Ising model on a k x l grid.  Two
gate sets share one code path:

  ZZ_X (default): bond gates exp(-i J dt Z(x)Z), site gates exp(-i h dt X),
                  observable Z at the chosen site.
  XX_Z (the paper's Eq. 1 convention): bond gates exp(-i J dt X(x)X), site
                  gates exp(-i h dt Z).  With the paper's R(theta) =
                  exp(-i theta P / 2), R_xx(2 J dt) = exp(-i J dt XX) and the two
                  R_z(h dt) factors of Eq. 6 are exp(-i (h dt / 2) Z) each.

Schedule of one step (Sec. 2.4, Eq. 6; reading: the paper calls Eq. 6 first
order although it is the symmetric split):
  order 1: all site gates with angle h dt, then bond colours 0, 1, 2, 3 with
           angle J dt;
  order 2: site gates with h dt / 2, colours 0..3 with J dt, site gates h dt / 2.

Every gate acts on the operator by O -> g^dagger O g (Eq. 5).

Pinned by: tests/test_oracle_dense.py (closed forms at J = 0 and h = 0, the
free-fermion solution of the chain).
"""
import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X2 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z2 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": X2, "Y": Y2, "Z": Z2}
PAULI_BY_INDEX = (I2, X2, Y2, Z2)   # p = 0:I, 1:X, 2:Y, 3:Z (Sec. 2.3)

GATESETS = {"ZZ_X": ("Z", "X"), "XX_Z": ("X", "Z")}


def rotation(P, angle):
    """exp(-i angle P) for a Pauli string P with P @ P = 1."""
    d = P.shape[0]
    return np.cos(angle) * np.eye(d, dtype=np.complex128) - 1j * np.sin(angle) * P


def bond_unitary(gateset, theta):
    p, _ = GATESETS[gateset]
    return rotation(np.kron(PAULI[p], PAULI[p]), theta)


def site_unitary(gateset, phi):
    _, q = GATESETS[gateset]
    return rotation(PAULI[q], phi)


def step_schedule(gateset, J, h, dt, order):
    """One Trotter step as a list of ('site', U2) and ('bond', colour, U4)."""
    if order not in (1, 2):
        raise ValueError("trotter order must be 1 or 2")
    bond = bond_unitary(gateset, J * dt)
    ops = []
    phi = h * dt if order == 1 else 0.5 * h * dt
    ops.append(("site", site_unitary(gateset, phi)))
    for c in range(4):
        ops.append(("bond", c, bond))
    if order == 2:
        ops.append(("site", site_unitary(gateset, phi)))
    return ops
