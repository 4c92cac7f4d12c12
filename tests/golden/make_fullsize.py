"""Write the oracle's expected values for the full-size parity tests
(tests/test_gpu_fullsize.py) to tests/golden/fullsize_10x10_chi100.txt.

Calls only the CPU oracle (``oracle/``) and the seeded input generator
(``workloads/synthetic.py``).  The workload is the 10x10, chi_max = 100
lattice of the benchmark (J = 1, h = 2, dt = 0.05, symmetric split, Z at
(3, 4), seed 0): every bond at chi_max, messages diag(lam), Gaussian site
tensors drawn in float32 (the precision the library stores them in).

1. Bond update (Sec. 2.5, Algorithm 1; Sec. 4.2 Eq. 10-12) of the colour-0
   bond (2, 4)-(3, 4), both sites interior (degree 4, m = chi^3 = 1e6 rows,
   n = 4 chi = 400 columns: the Cholesky-QR branch on the GPU), after the
   half-angle site gates that the symmetric split applies first (the GPU
   folds them into this bond gate).  Stored: the Vidal spectrum, the raw
   singular values around the cut, the norm of every slice k of the new bond
   leg of both new site tensors, and seeded samples of their Pauli
   coefficients (24 per slice k).
2. One damped double-layer BP sweep (Sec. 4.2 Eq. 13, Sec. 6.3 Eq. 19,
   alpha = 0.5) from the synthetic messages: the messages that the interior
   site (3, 4), the edge site (0, 4) and the corner (0, 0) send.  Stored:
   each message's diagonal and 400 seeded off-diagonal entries.

The sha256 of each input site tensor (float32 bytes) is stored so that the
test can tell a changed input generator from a wrong result.

Usage: python tests/golden/make_fullsize.py   (about ten minutes, ~45 GB RAM)
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import bp as obp  # noqa: E402
from oracle import gates as og  # noqa: E402
from oracle import pepo as opepo  # noqa: E402
from workloads.synthetic import bond_data, site_tensor  # noqa: E402

OUT = os.path.join(HERE, "fullsize_10x10_chi100.txt")
W = dict(Lx=10, Ly=10, J=1.0, h=2.0, dt=0.05, chi=100, obs=(3, 4), seed=0, alpha=0.5,
         eps_cut=1e-11, pinv_rel=1e-12)
BOND = (42, 43)              # sites (2, 4) and (3, 4); bond id 4 * 9 + 2 = 38, colour 0
BP_SITES = (43, 40, 0)       # interior (3, 4), edge (0, 4), corner (0, 0)
SAMPLES_PER_SLICE = 24
OFFDIAG_SAMPLES = 400


def inputs(sites):
    Lx, Ly, chi = W["Lx"], W["Ly"], W["chi"]
    return {v: site_tensor(Lx, Ly, chi, W["seed"], v, np.float32, obs=W["obs"]) for v in sites}


def sha(t):
    return hashlib.sha256(np.ascontiguousarray(t).tobytes()).hexdigest()


def to_pauli(O):
    """Pauli coefficients psi[..., p] = Tr(P_p O) / 2 of a 2x2 operator block."""
    P = np.stack(og.PAULI_BY_INDEX)
    c = np.einsum("...ab,pba->...p", O, P) / 2.0
    return c


def main():
    Lx, Ly, chi = W["Lx"], W["Ly"], W["chi"]
    bd = bond_data(Lx, Ly, chi)
    lines = ["# Oracle values for the 10x10 chi_max = 100 full-size parity tests.",
             "# Written by tests/golden/make_fullsize.py (calls oracle/ and workloads/ only).",
             "# config " + " ".join("%s=%s" % (k, W[k]) for k in sorted(W))]
    # ---- 1. bond update of bond (42, 43)
    t0 = time.time()
    raw = inputs(BOND)
    for v in BOND:
        lines.append("input %d %s" % (v, sha(raw[v])))
    sites = {v: raw[v].astype(np.float64) for v in BOND}
    del raw
    net = opepo.from_pauli(Lx, Ly, W["obs"], "Z", sites, bd["chi"], bd["msgs"], sites_subset=set(BOND))
    del sites
    g1 = og.site_unitary("ZZ_X", 0.5 * W["h"] * W["dt"])
    g2 = og.bond_unitary("ZZ_X", W["J"] * W["dt"])
    for v in BOND:
        opepo.apply_site_gate(net, v, g1)
    r = opepo.bond_update(net, BOND[0], BOND[1], g2, chi, W["eps_cut"], W["pinv_rel"])
    print("bond update %.1f s, chi_new %d" % (time.time() - t0, r["chi"]), file=sys.stderr, flush=True)
    s = r["s"]
    lines.append("lam %d %s" % (len(r["lam"]), " ".join("%.17g" % x for x in r["lam"])))
    lines.append("s %d %s" % (min(len(s), chi + 2), " ".join("%.17g" % x for x in s[:chi + 2])))
    rng = np.random.default_rng(12345)
    for v, other in (BOND, BOND[::-1]):
        psi = to_pauli(net.O[v])
        net.O[v] = None
        imag = float(np.max(np.abs(psi.imag)))
        psi = np.ascontiguousarray(psi.real)
        ax = net.axis(v, other)
        lines.append("imag %d %.3e" % (v, imag))
        norms = np.sqrt(np.sum(np.moveaxis(psi, ax, 0).reshape(psi.shape[ax], -1) ** 2, axis=1))
        lines.append("colnorm %d %d %s" % (v, ax, " ".join("%.17g" % x for x in norms)))
        shape = psi.shape
        for k in range(shape[ax]):
            for _ in range(SAMPLES_PER_SLICE):
                idx = [int(rng.integers(0, n)) for n in shape]
                idx[ax] = k
                lines.append("sample %d %s %.17g" % (v, " ".join(str(i) for i in idx), psi[tuple(idx)]))
        del psi
    del net
    # ---- 2. one damped BP sweep: messages sent by BP_SITES
    t0 = time.time()
    raw = inputs(BP_SITES)
    for v in BP_SITES:
        lines.append("input %d %s" % (v, sha(raw[v])))
    sites = {v: raw[v].astype(np.float64) for v in BP_SITES}
    del raw
    net = opepo.from_pauli(Lx, Ly, W["obs"], "Z", sites, bd["chi"], bd["msgs"], sites_subset=set(BP_SITES))
    del sites
    bid = {}
    for b, (a, c) in enumerate(_bonds(Lx, Ly)):
        bid[(a, c)] = (b, 0)
        bid[(c, a)] = (b, 1)
    for v in BP_SITES:
        for k, (_, u) in enumerate(net.legs[v]):
            Mn, _ = obp.double_update(net, v, k, net.M, W["alpha"])
            Mn = np.real(Mn)
            b, d = bid[(v, u)]
            n = Mn.shape[0]
            lines.append("msgdiag %d %d %d %s" % (b, d, n, " ".join("%.17g" % x for x in np.diag(Mn))))
            for _ in range(OFFDIAG_SAMPLES):
                i, j = int(rng.integers(0, n)), int(rng.integers(0, n))
                lines.append("msg %d %d %d %d %.17g" % (b, d, i, j, Mn[i, j]))
            print("message %d -> %d done (%.1f s)" % (v, u, time.time() - t0), file=sys.stderr, flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


def _bonds(Lx, Ly):
    out = []
    for y in range(Ly):
        for x in range(Lx - 1):
            out.append((y * Lx + x, y * Lx + x + 1))
    for y in range(Ly - 1):
        for x in range(Lx):
            out.append((y * Lx + x, (y + 1) * Lx + x))
    return out


if __name__ == "__main__":
    main()
