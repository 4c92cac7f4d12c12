"""BP trap remediation (Sec. 6.3).

On loopy grids damped BP can settle in a wrong fixed point.  The paper's
procedure after each measured layer:
  1. a layer whose BP converged but needed 30 or more sweeps is a candidate
     Type-1 trap (`trap_type1`);
  2. it is confirmed when C fell below half of the previous layer's value
     while the discarded weight did not jump (`c_drop`, pepo_c_drop);
  3. BP is run again with another damping, from the messages it started from;
  4. if every damping is trapped, the bond dimension is too small: raise chi
     rather than tune the damping.
Here the retries follow `alphas` in order, skipping the damping in force.
When every retry is trapped the layer is measured once more with the
original damping from the same start, so the device state and the returned
record are those of the unremediated run, and `increase_chi` is set.

Only whole-context BP runs exist (pepo_bp_converge converges every instance),
so the remediation handles one-instance contexts.
"""
from . import PepoError

ALPHAS = (0.5, 0.8, 1.0)


def measure(eng, inst=0, alphas=ALPHAS, require_c_drop=True):
    """Double-layer BP and the correlator with remediation.  Returns
    (C, diag, info); info = {"trapped", "alpha", "retries", "increase_chi"}."""
    if eng.n_inst != 1:
        raise PepoError("trap remediation handles one-instance contexts")
    alpha0, tol, max_sweeps = eng.bp_params(inst)
    start = eng.get_messages(inst)
    eng.bp_converge()
    C, D = eng.correlator()
    d = D[inst]
    info = {"trapped": False, "alpha": alpha0, "retries": [], "increase_chi": False}
    if not (d["trap_type1"] and (d["c_drop"] or not require_c_drop)):
        return C[inst], d, info
    info["trapped"] = True
    try:
        for a in alphas:
            if a == alpha0:
                continue
            eng.set_bp_params(a, tol, max_sweeps, inst)
            eng.set_messages(start, inst)
            eng.bp_converge()
            C2, D2 = eng.correlator()
            d2 = D2[inst]
            info["retries"].append({"alpha": a, "C": C2[inst], "bp_sweeps": d2["bp_sweeps"],
                                    "trap_type1": d2["trap_type1"]})
            if not d2["trap_type1"]:
                info["alpha"] = a
                return C2[inst], d2, info
        info["increase_chi"] = True
    finally:
        eng.set_bp_params(alpha0, tol, max_sweeps, inst)
    eng.set_messages(start, inst)
    eng.bp_converge()
    C, D = eng.correlator()
    return C[inst], D[inst], info
