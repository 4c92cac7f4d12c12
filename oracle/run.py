"""The oracle's time loop (Fig. 1 pipeline: gates, BP, measure).

Per step: the Trotter schedule of ``gates.step_schedule`` (site gates applied
separately, never folded into bond gates), bond colours 0..3, then
double-layer BP from the current messages (diag(lam) after the gates), then
single-layer BP and the Bethe value of C(t).  Step 0 measures the initial
network the same way.

Each record holds: t, C, C_proj, norm (Bethe norm), bp sweeps / delta (both
layers), gate_err (Table 1: discarded weight summed over the step's bonds),
and per bond its chi and lam.
"""
import numpy as np

from . import gates as G
from .bp import bethe, bp_double, bp_single, pinned_tensors
from .lattice import bonds_by_colour
from .pepo import Network, apply_site_gates, bond_key, bond_update

DEFAULTS = dict(J=1.0, h=1.0, dt=0.05, order=1, obs=None, obs_pauli="Z", chi_max=8,
                eps_cut=1e-11, bp_alpha=0.5, bp_tol=1e-5, bp_max_sweeps=100,
                gateset="ZZ_X", pinv_rel=1e-12, nsteps=1)


def full_config(cfg):
    c = dict(DEFAULTS)
    c.update(cfg)
    if c["obs"] is None:
        c["obs"] = ((c["Lx"] - 1) // 2, (c["Ly"] - 1) // 2)
    return c


def measure(net, c):
    sw2, d2 = bp_double(net, c["bp_alpha"], c["bp_tol"], c["bp_max_sweeps"])
    t = pinned_tensors(net)
    m, sw1, d1 = bp_single(net, t, c["bp_alpha"], c["bp_tol"], c["bp_max_sweeps"])
    b = bethe(net, t, m, net.M)
    b.update(bp_sweeps=sw2, bp_delta=d2, bp1_sweeps=sw1, bp1_delta=d1)
    return b


def trotter_step(net, c, record=None):
    sched = G.step_schedule(c["gateset"], c["J"], c["h"], c["dt"], c["order"])
    colours = bonds_by_colour(net.Lx, net.Ly)
    gate_err = 0.0
    for op in sched:
        if op[0] == "site":
            apply_site_gates(net, op[1])
        else:
            for (v1, v2, _, _) in colours[op[1]]:
                r = bond_update(net, v1, v2, op[2], c["chi_max"], c["eps_cut"], c["pinv_rel"])
                gate_err += r["disc"]
                if record is not None:
                    record.append((v1, v2, r))
    return gate_err


def simulate(cfg, nsteps=None, net=None):
    c = full_config(cfg)
    n = c["nsteps"] if nsteps is None else nsteps
    if net is None:
        net = Network(c["Lx"], c["Ly"], c["obs"], c["obs_pauli"])
    out = []
    r0 = measure(net, c)
    r0.update(t=0.0, gate_err=0.0, chi={}, lam={})
    out.append(r0)
    for step in range(1, n + 1):
        rec = []
        ge = trotter_step(net, c, rec)
        r = measure(net, c)
        r.update(t=step * c["dt"], gate_err=ge,
                 chi={bond_key(a, b): x["chi"] for (a, b, x) in rec},
                 lam={bond_key(a, b): x["lam"] for (a, b, x) in rec})
        out.append(r)
    return out, net
