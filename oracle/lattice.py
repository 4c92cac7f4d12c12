"""Square-lattice geometry used by the oracle.

Sites are (x, y) with x = column, y = row, origin at the top-left; the linear
index is v = y * Lx + x.  Each site lists its legs in the canonical order
[U, D, L, R] (Sec. 3.1 "GPU Tensor Permutation": canonical bond order
[U, D, L, R, Pauli]), skipping legs that fall off the open boundary
(Sec. 2.1, open boundary conditions).

The bonds are split into four colour classes such that no two bonds of one
class share a site (Sec. 2.4, four-colour decomposition):
  colour 0: horizontal bonds (x, y)-(x+1, y) with x even
  colour 1: horizontal bonds with x odd
  colour 2: vertical bonds (x, y)-(x, y+1) with y even
  colour 3: vertical bonds with y odd
The paper does not fix the colour order; the oracle applies colours 0,1,2,3.

Pinned by: tests/test_oracle_dense.py (h = 0 closed forms depend on the number
of bonds at the observable site) and the chain/tree tests.
"""

LEGS = ("U", "D", "L", "R")
OPPOSITE = {"U": "D", "D": "U", "L": "R", "R": "L"}


def site_index(x, y, Lx):
    return y * Lx + x


def site_coords(v, Lx):
    return v % Lx, v // Lx


def legs_of(x, y, Lx, Ly):
    """Present legs of site (x, y) in canonical order, with the neighbour index."""
    out = []
    if y > 0:
        out.append(("U", site_index(x, y - 1, Lx)))
    if y < Ly - 1:
        out.append(("D", site_index(x, y + 1, Lx)))
    if x > 0:
        out.append(("L", site_index(x - 1, y, Lx)))
    if x < Lx - 1:
        out.append(("R", site_index(x + 1, y, Lx)))
    return out


def bonds_by_colour(Lx, Ly):
    """Four lists of bonds (v1, v2, leg_of_v1, leg_of_v2)."""
    colours = [[], [], [], []]
    for y in range(Ly):
        for x in range(Lx - 1):
            colours[x % 2].append((site_index(x, y, Lx), site_index(x + 1, y, Lx), "R", "L"))
    for y in range(Ly - 1):
        for x in range(Lx):
            colours[2 + (y % 2)].append((site_index(x, y, Lx), site_index(x, y + 1, Lx), "D", "U"))
    return colours


def all_bonds(Lx, Ly):
    return [b for c in bonds_by_colour(Lx, Ly) for b in c]
