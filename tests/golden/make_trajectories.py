"""Write oracle C(t) trajectories used as stored expected values by the GPU tests.

Calls only the CPU oracle (``oracle/``).  Each case is evolved step by step;
after every step one line (t, C, C_proj, log of the Bethe norm, double- and
single-layer BP sweeps, discarded weight) is appended and flushed, so a run
that is stopped early leaves a usable prefix.  At the end the Vidal
spectrum of every bond is written, in the library's bond numbering.

Usage: python tests/golden/make_trajectories.py CASE [NSTEPS]
Cases:
  c2_chi20, c2_chi40, c2_chi60   4x4, J = 1, h = 2, Z at (1, 1), second-order
                                 split, dt = 0.05, ZZ / X gates (40 steps = t 2)
  paper4x4_chi40                 the paper's convention on 4x4 (XX / Z gates,
                                 h = J = -1, dt = 0.1, Z at (1, 1)), 20 steps
  c4_chi64                       8x8, J = 1, h = 2, Z at (3, 3), second-order
                                 split, dt = 0.05, chi_max = 64 (the prefix the
                                 oracle finishes)
Output: tests/golden/traj_<CASE>.txt
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.run import full_config, measure, trotter_step  # noqa: E402
from oracle.pepo import Network, bond_key  # noqa: E402

C2 = dict(Lx=4, Ly=4, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), obs_pauli="Z", eps_cut=1e-11,
          bp_alpha=0.5, bp_tol=1e-5, bp_max_sweeps=100, gateset="ZZ_X", pinv_rel=1e-12)
# the paper's own convention (Sec. 6): XX / Z gates, h = J = -1, dt = 0.1,
# symmetric split, Z at (1, 1) of the 4x4 grid
PAPER_4X4 = dict(Lx=4, Ly=4, J=-1.0, h=-1.0, dt=0.1, order=2, obs=(1, 1), obs_pauli="Z", eps_cut=1e-11,
                 bp_alpha=0.5, bp_tol=1e-5, bp_max_sweeps=100, gateset="XX_Z", pinv_rel=1e-12)
CASES = {
    "c2_chi20": dict(C2, chi_max=20, nsteps=40),
    "c2_chi40": dict(C2, chi_max=40, nsteps=40),
    "c2_chi60": dict(C2, chi_max=60, nsteps=40),
    "paper4x4_chi40": dict(PAPER_4X4, chi_max=40, nsteps=20),
    "c4_chi64": dict(C2, Lx=8, Ly=8, obs=(3, 3), chi_max=64, nsteps=24),
}


def bond_ids(Lx, Ly):
    """(a, b) -> library bond id (horizontal y*(Lx-1)+x first, then vertical)."""
    out = {}
    for y in range(Ly):
        for x in range(Lx - 1):
            out[(y * Lx + x, y * Lx + x + 1)] = y * (Lx - 1) + x
    for y in range(Ly - 1):
        for x in range(Lx):
            out[(y * Lx + x, (y + 1) * Lx + x)] = Ly * (Lx - 1) + y * Lx + x
    return out


def main():
    name = sys.argv[1]
    case = dict(CASES[name])
    nsteps = int(sys.argv[2]) if len(sys.argv) > 2 else case.pop("nsteps")
    case.pop("nsteps", None)
    c = full_config(case)
    path = os.path.join(HERE, "traj_%s.txt" % name)
    net = Network(c["Lx"], c["Ly"], c["obs"], c["obs_pauli"])
    with open(path, "w") as f:
        f.write("# oracle trajectory %s, written by tests/golden/make_trajectories.py (oracle only)\n" % name)
        f.write("# config %s\n" % " ".join("%s=%s" % (k, c[k]) for k in sorted(c) if k != "nsteps"))
        f.write("# step t C C_proj log_norm bp_sweeps bp1_sweeps gate_err seconds\n")
        t0 = time.time()
        r = measure(net, c)
        f.write("%d %.4f %.17g %.17g %.17g %d %d %.17g %.1f\n" % (0, 0.0, r["C"], r["C_proj"], r["log_norm"],
                                                                   r["bp_sweeps"], r["bp1_sweeps"], 0.0,
                                                                   time.time() - t0))
        f.flush()
        for step in range(1, nsteps + 1):
            t0 = time.time()
            ge = trotter_step(net, c)
            r = measure(net, c)
            f.write("%d %.4f %.17g %.17g %.17g %d %d %.17g %.1f\n" % (step, step * c["dt"], r["C"], r["C_proj"],
                                                                       r["log_norm"], r["bp_sweeps"],
                                                                       r["bp1_sweeps"], ge, time.time() - t0))
            f.flush()
            print(name, step, r["C"], "%.1f s" % (time.time() - t0), file=sys.stderr, flush=True)
        f.write("# lam bond chi values...  (Vidal spectra after the last step)\n")
        for (a, b), k in sorted(bond_ids(c["Lx"], c["Ly"]).items(), key=lambda x: x[1]):
            lam = net.lam[bond_key(a, b)]
            f.write("lam %d %d %s\n" % (k, len(lam), " ".join("%.17g" % x for x in lam)))


if __name__ == "__main__":
    main()
