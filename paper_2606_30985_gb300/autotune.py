"""Launch-shape autotuner for the Gram kernels (batching and autotuning; the
paper has no counterpart).

The K range of a Gram is cut into splits that are reduced in FP64 afterwards
(pepo_set_tuning).  How many splits fill the GPU best depends on the bond
dimension (the size of each Gram) and on the precision mode (SIMT or tensor
core kernels).  `sweep` times, per (chi class, precision), one Trotter step and
a fixed number of double-layer BP sweeps on a seeded synthetic saturated state
for each candidate split count, using the library's per-kernel-class timers
(CUDA events around each launch), and caches the fastest counts in a JSON file.
`lookup` returns the cached shapes of the nearest class; Engine applies them
at construction (Engine(..., tuning="cache")).

Run on the target GPU from the repository root:
    python -m paper_2606_30985_gb300.autotune --chis 16 32 48 64 100
"""
import argparse
import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
LEG_SPLITS = (16, 32, 64, 96, 128)     # free-leg Gram (pepo_set_tuning bounds: 1..128)
ROWS_SPLITS = (8, 16, 32, 64)          # Cholesky-QR Gram (bounds: 1..64)


def load(path=CACHE):
    """The cached table ({"version": 1, "classes": [...]}), or None."""
    if not path or not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    if not isinstance(table, dict) or table.get("version") != 1:
        return None
    return table


def lookup(chi_max, precision, path=CACHE, table=None):
    """Launch shapes cached for the class nearest to (chi_max, precision): the
    smallest cached chi >= chi_max, else the largest cached chi; None when
    nothing is cached for that precision."""
    table = table if table is not None else load(path)
    if not table:
        return None
    recs = [r for r in table.get("classes", []) if r.get("precision") == precision]
    if not recs:
        return None
    above = [r for r in recs if r["chi_max"] >= chi_max]
    rec = min(above, key=lambda r: r["chi_max"]) if above else max(recs, key=lambda r: r["chi_max"])
    return {"gram_leg_splits": int(rec["gram_leg_splits"]), "gram_rows_splits": int(rec["gram_rows_splits"])}


def _upload(eng, Lx, Ly, chi, obs, seed):
    import numpy as np
    from workloads.synthetic import bond_data, site_tensor
    bd = bond_data(Lx, Ly, chi)
    eng.set_bonds(0, bd["chi"], bd["lam"], bd["msgs"])
    for v in range(Lx * Ly):
        eng.set_site(0, v, site_tensor(Lx, Ly, chi, seed, v, np.float32, obs=obs))


def measure(eng, snap, leg_splits, rows_splits, reps):
    """Best-of-reps milliseconds of the free-leg Gram and of the Cholesky-QR
    Gram (each with its split reduction) over one Trotter step and the BP
    sweeps that follow, starting every repetition from the snapshot."""
    eng.set_tuning(leg_splits, rows_splits)
    best_leg = best_rows = float("inf")
    for _ in range(reps):
        eng.load_state(snap)
        eng.reset_timing()
        eng.trotter_step(1)
        eng.bp_converge()
        t = eng.timing()
        best_leg = min(best_leg, t["gram_leg"]["ms"] + t["gram_leg_reduce"]["ms"])
        best_rows = min(best_rows, t["gram_rows"]["ms"] + t["gram_rows_reduce"]["ms"])
    return best_leg, best_rows


def sweep(chis=(16, 32, 48, 64, 100), precisions=("tf32x3",), grid=4, bp_sweeps=3, reps=2, path=CACHE,
          seed=11, leg_candidates=LEG_SPLITS, rows_candidates=ROWS_SPLITS, log=print):
    """Time every candidate split count per (chi, precision) class on a
    grid x grid synthetic saturated state and merge the winners into the JSON
    cache at `path` (None: do not write).  Returns the table."""
    import torch
    import paper_2606_30985_gb300 as pkg
    table = load(path) or {"version": 1, "classes": []}
    device = torch.cuda.get_device_name()
    for prec in precisions:
        for chi in chis:
            cfg = pkg.Config(Lx=grid, Ly=grid, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=chi,
                             precision=prec, bp_max_sweeps=bp_sweeps)
            eng = pkg.Engine(cfg, tuning=None)
            try:
                _upload(eng, grid, grid, chi, (1, 1), seed)
                snap = torch.empty(eng.state_bytes(), dtype=torch.uint8, device="cuda")
                eng.save_state(snap)
                eng.set_timing(True)
                leg = {s: measure(eng, snap, s, 0, reps)[0] for s in leg_candidates}
                rows = {s: measure(eng, snap, 0, s, reps)[1] for s in rows_candidates}
            finally:
                eng.close()
            rec = {"chi_max": chi, "precision": prec, "grid": grid, "bp_sweeps": bp_sweeps, "device": device,
                   "gram_leg_splits": min(leg, key=leg.get), "gram_rows_splits": min(rows, key=rows.get),
                   "gram_leg_ms": {str(k): round(v, 4) for k, v in leg.items()},
                   "gram_rows_ms": {str(k): round(v, 4) for k, v in rows.items()}}
            table["classes"] = [r for r in table["classes"]
                                if not (r["chi_max"] == chi and r["precision"] == prec)] + [rec]
            if log:
                log("chi %d %s: gram_leg splits %d (%s ms), gram_rows splits %d (%s ms)" % (
                    chi, prec, rec["gram_leg_splits"], rec["gram_leg_ms"], rec["gram_rows_splits"],
                    rec["gram_rows_ms"]))
    table["classes"].sort(key=lambda r: (r["precision"], r["chi_max"]))
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    return table


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--chis", type=int, nargs="+", default=[16, 32, 48, 64, 100])
    ap.add_argument("--prec", nargs="+", default=["tf32x3"])
    ap.add_argument("--grid", type=int, default=4)
    ap.add_argument("--bp-sweeps", type=int, default=3)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=CACHE)
    a = ap.parse_args()
    sweep(tuple(a.chis), tuple(a.prec), a.grid, a.bp_sweeps, a.reps, a.out)


if __name__ == "__main__":
    main()
