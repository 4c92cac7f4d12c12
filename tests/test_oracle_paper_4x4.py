"""Pin of the whole oracle (gates, bond updates with truncation, loopy BP and
the Bethe value) against C(t) values the paper prints for the 4x4 grid.

Sec. 6.2 gives the chi ladder of the 4x4 grid at t = 2.0, 0.0572 at chi = 40,
and Table mi60_chi prints the same point from the paper's second GPU
implementation (0.0577; the two agree within 1e-3 at this trap-free operating
point).  Sec. 6.4's table gives C(1.4) = 0.085 on 4x4, where the paper finds
every chi >= 40 in agreement.  On this grid the Bethe estimate departs from
the exact dynamics (typicality on the 16-qubit grid: C(1.4) = 0.0908,
C(2.0) = 0.0645), so these values check the loopy BP and the Bethe ratio, not
only the gates.  Convention of Sec. 6: XX / Z gates, h = J = -1, dt = 0.1,
the symmetric split, Z at (1, 1), eps_cut = 1e-11; the BP settings are the
oracle's defaults (damping 0.5, tolerance 1e-5, 100 sweeps).

Measured with this test's configuration: C(1.4) = 0.08533, C(2.0) = 0.05715.
About 80 minutes on 8 host cores: marked slow (pytest --runslow).

The default run pins the loopy part too, at t = 1.4 only and chi = 20
(14 steps, a few minutes): the oracle's ladder there is C(1.4) = 0.08794
(chi 12), 0.08714 (16), 0.08570 (20), 0.08533 (40), so chi = 20 is within
4e-4 of chi = 40 and within the pin's 1e-3 of the printed 0.085, while the
exact dynamics (0.0908) is 5.8e-3 away: a mistake in the loopy Bethe ratio
or in the message normalisation moves the value far beyond the bound.
"""
import os

import pytest

from oracle.run import simulate

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ct_4x4_chi40.txt")
TOL = 1e-3   # print rounding (5e-4) and the paper's 1e-3 spread between its two implementations


def printed_values():
    """{step: [values]} from the fixture (t = step * 0.1)."""
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            t, v = s.split()[:2]
            out.setdefault(int(round(float(t) / 0.1)), []).append(float(v))
    return out


def test_4x4_chi20_matches_the_printed_value_at_t14():
    want = printed_values()[14]
    cfg = dict(Lx=4, Ly=4, J=-1.0, h=-1.0, dt=0.1, order=2, obs=(1, 1), chi_max=20, eps_cut=1e-11,
               gateset="XX_Z", obs_pauli="Z")
    recs, _ = simulate(cfg, nsteps=14)
    for v in want:
        assert abs(recs[14]["C"] - v) < TOL, (recs[14]["C"], v)


@pytest.mark.slow
def test_4x4_chi40_matches_the_printed_values():
    want = printed_values()
    assert sorted(want) == [14, 20]
    # BP runs after every step, as in the method: its messages are the
    # environments of the next step's bond updates
    cfg = dict(Lx=4, Ly=4, J=-1.0, h=-1.0, dt=0.1, order=2, obs=(1, 1), chi_max=40, eps_cut=1e-11,
               gateset="XX_Z", obs_pauli="Z")
    recs, _ = simulate(cfg, nsteps=max(want))
    for step, values in want.items():
        for v in values:
            assert abs(recs[step]["C"] - v) < TOL, (step, recs[step]["C"], v)
