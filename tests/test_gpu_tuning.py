"""Launch-shape tuning (pepo_set_tuning) and the autotuner sweep on the GPU."""
import json

import pytest

import paper_2606_30985_gb300 as pkg
from paper_2606_30985_gb300 import autotune

pytestmark = pytest.mark.gpu

CFG = dict(Lx=4, Ly=4, J=1.0, h=1.5, dt=0.05, order=2, obs=(1, 1), chi_max=8)


def _run(eng, steps=4):
    out = []
    for _ in range(steps):
        eng.trotter_step(1)
        sw, _ = eng.bp_converge()
        C, _ = eng.correlator()
        out.append((C[0], sw[0]))
    return out


def test_tuning_round_trip_and_bounds():
    eng = pkg.Engine(pkg.Config(precision="fp32", **CFG), tuning=None)
    assert eng.get_tuning() == {"gram_leg_splits": 64, "gram_rows_splits": 32}
    eng.set_tuning(16, 8)
    assert eng.get_tuning() == {"gram_leg_splits": 16, "gram_rows_splits": 8}
    for bad in ((0, 65), (129, 0), (-1, 0)):
        with pytest.raises(pkg.PepoError):
            eng.set_tuning(*bad)
    assert eng.get_tuning() == {"gram_leg_splits": 16, "gram_rows_splits": 8}   # unchanged on error
    eng.set_tuning(0, 0)
    assert eng.get_tuning() == {"gram_leg_splits": 64, "gram_rows_splits": 32}
    eng.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("tf32x3", 1e-6)])
def test_split_counts_change_only_rounding(precision, tol):
    a = pkg.Engine(pkg.Config(precision=precision, **CFG), tuning=None)
    ra = _run(a)
    a.close()
    b = pkg.Engine(pkg.Config(precision=precision, **CFG), tuning={"gram_leg_splits": 3, "gram_rows_splits": 5})
    rb = _run(b)
    # change the shapes mid-run too (captured graphs are dropped and recaptured)
    b.set_tuning(128, 64)
    rb += _run(b, 2)
    b.close()
    c = pkg.Engine(pkg.Config(precision=precision, **CFG), tuning=None)
    rc = _run(c, 6)
    c.close()
    assert len(rb) == len(rc)
    for (Ca, sa), (Cb, sb) in zip(ra + rc[4:], rb):
        assert abs(Ca - Cb) <= tol * max(1.0, abs(Ca))
        assert sa == sb


def test_sweep_writes_a_cache_the_engine_applies(tmp_path):
    path = str(tmp_path / "tuning.json")
    table = autotune.sweep(chis=(6,), precisions=("tf32x3",), grid=3, bp_sweeps=2, reps=1, path=path,
                           leg_candidates=(8, 64), rows_candidates=(4, 32), log=None)
    rec = table["classes"][0]
    assert rec["gram_leg_splits"] in (8, 64) and rec["gram_rows_splits"] in (4, 32)
    assert set(rec["gram_leg_ms"]) == {"8", "64"} and all(v > 0 for v in rec["gram_leg_ms"].values())
    with open(path) as f:
        assert json.load(f) == table
    want = autotune.lookup(6, "tf32x3", path)
    eng = pkg.Engine(pkg.Config(precision="tf32x3", Lx=3, Ly=3, chi_max=6), tuning=want)
    assert eng.get_tuning() == want
    eng.close()
