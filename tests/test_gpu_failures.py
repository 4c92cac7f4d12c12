"""Failure handling on the GPU, in forms that fault and hang nothing.

* The Sec. 6.3 / Table 1 trap signals from the device state: a sweep budget
  of one (Type 2), slow damped convergence (Type 1, 30 sweeps or more), and
  the C-collapse check across layers (closed form C(t) = cos(2 h t) at J = 0,
  where |C| falls below half of the previous layer's with no discarded
  weight), including its reset by a state restore.
* A non-finite coefficient uploaded from the host reaches BP and the
  correlator and is reported in flags bit 1, not raised.
* The BP settings and message snapshots of the trap remediation act on the
  device: a message round trip restarts BP from the same messages (same sweeps,
  same messages), and undamped BP from them matches the oracle's.
* The wait limit of the tensor-core pipelines: set to 1 ns, the first wait
  that is not already satisfied runs out, the kernels return, the next call
  that reads results fails with PEPO_E_CUDA, and after the limit is restored
  and the state reloaded the context gives the undisturbed result.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import bp as obp
from oracle import pepo as opepo

pytestmark = pytest.mark.gpu


def config(**kw):
    base = dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, chi_max=8, precision="fp32")
    base.update(kw)
    return pkg.Config(**base)


def test_sweep_budget_of_one_sets_trap_type2():
    eng = pkg.Engine(config())
    try:
        eng.trotter_step(3)
        eng.set_bp_params(0.5, tol=1e-14, max_sweeps=1)
        sw, de = eng.bp_converge()
        assert sw == [1] and de[0] > 1e-14
        _, D = eng.correlator()
        assert D[0]["bp_sweeps"] == 1
        assert D[0]["trap_type2"] == 1 and D[0]["trap_type1"] == 0
    finally:
        eng.close()


def test_slow_damping_sets_trap_type1():
    eng = pkg.Engine(config())
    try:
        eng.trotter_step(3)
        eng.set_bp_params(0.02, tol=1e-6, max_sweeps=2000)
        sw, de = eng.bp_converge()
        assert 30 <= sw[0] < 2000 and de[0] < 1e-6
        _, D = eng.correlator()
        assert D[0]["trap_type1"] == 1 and D[0]["trap_type2"] == 0
    finally:
        eng.close()


def test_c_drop_across_layers_and_after_restore():
    import torch
    # J = 0: C(t) = cos(2 h t) exactly, every chi stays 1, nothing is discarded.
    # h dt = 0.35: C = cos(0.7) = 0.765 after one step, cos(1.4) = 0.170 after two
    eng = pkg.Engine(config(J=0.0, h=7.0, chi_max=4))
    try:
        recs = eng.run(2)
        C = np.array([r["C"] for r in recs])
        assert np.max(np.abs(C - np.cos(2 * 7.0 * 0.05 * np.arange(3)))) < 1e-6
        assert [r["c_drop"] for r in recs] == [0, 0, 1]
        assert all(r["gate_err"] < 1e-12 for r in recs)
        # a repeated measurement of the same layer keeps the layer before it
        eng.bp_converge()
        _, D = eng.correlator()
        assert D[0]["c_drop"] == 1
        # a restore forgets the previous layer: no drop until a new one is measured
        snap = torch.empty(eng.state_bytes(), dtype=torch.uint8, device="cuda:0")
        eng.save_state(snap)
        eng.load_state(snap)
        eng.bp_converge()
        _, D = eng.correlator()
        assert D[0]["c_drop"] == 0 and D[0]["steps"] == 2
    finally:
        eng.close()


def test_nonfinite_site_sets_flag_bit1():
    eng = pkg.Engine(config(chi_max=4))
    try:
        eng.trotter_step(2)
        eng.bp_converge()
        _, D = eng.correlator()
        assert D[0]["flags"] & 2 == 0
        t, _ = eng.site(0, 4)
        t = np.array(t)
        t.flat[5] = np.nan
        eng.set_site(0, 4, t)
        eng.set_bp_params(0.5, tol=1e-5, max_sweeps=5)
        eng.bp_converge()
        _, D = eng.correlator()
        assert D[0]["flags"] & 2, D[0]["flags"]
    finally:
        eng.close()


def test_bp_settings_and_message_round_trip_on_the_device():
    cfg = config(Lx=4, Ly=4, h=2.0, obs=(1, 1), order=2, chi_max=8)
    eng = pkg.Engine(cfg)
    try:
        eng.trotter_step(4)
        M0 = eng.get_messages()
        sw_a, _ = eng.bp_converge()
        Ma = eng.get_messages()
        eng.set_messages(M0)
        assert np.array_equal(eng.get_messages(), M0)
        eng.set_bp_params(1.0)
        sw_b, _ = eng.bp_converge()
        Mb = eng.get_messages()
        eng.set_messages(M0)
        eng.set_bp_params(0.5)
        sw_c, _ = eng.bp_converge()
        Mc = eng.get_messages()
        assert sw_c == sw_a and np.array_equal(Mc, Ma)
        assert sw_b != sw_a
        # undamped BP from M0 on the same network, run by the oracle
        nb = eng.num_bonds()
        chi = [len(eng.spectrum(0, b)) for b in range(nb)]
        sites = [eng.site(0, v)[0] for v in range(cfg.Lx * cfg.Ly)]
        msgs = M0.reshape(nb, 2, cfg.chi_max, cfg.chi_max)
        net = opepo.from_pauli(cfg.Lx, cfg.Ly, cfg.obs, "Z", sites, chi, msgs)
        obp.bp_double(net, 1.0, cfg.bp_tol, cfg.bp_max_sweeps)
        ref = opepo.from_pauli(cfg.Lx, cfg.Ly, cfg.obs, "Z", sites, chi,
                               Mb.reshape(nb, 2, cfg.chi_max, cfg.chi_max))
        err = max(float(np.max(np.abs(net.M[k] - ref.M[k]))) for k in net.M)
        assert err < 1e-4, err
    finally:
        eng.close()


def test_wait_limit_expiry_is_reported_and_the_context_recovers():
    import torch
    eng = pkg.Engine(config(precision="tf32x3"))
    try:
        eng.trotter_step(3)
        snap = torch.empty(eng.state_bytes(), dtype=torch.uint8, device="cuda:0")
        eng.save_state(snap)
        eng.trotter_step(1)
        eng.bp_converge()
        C_ref, _ = eng.correlator()
        eng.load_state(snap)
        eng.set_wait_limit(1e-9)
        raised = None
        for _ in range(3):
            try:
                eng.trotter_step(1)
                eng.bp_converge()
            except pkg.PepoError as e:
                raised = str(e)
                break
        assert raised is not None and "wait limit" in raised, raised
        eng.set_wait_limit(4.0)
        eng.load_state(snap)
        eng.trotter_step(1)
        eng.bp_converge()
        C, D = eng.correlator()
        assert abs(C[0] - C_ref[0]) < 1e-9, (C, C_ref)
        assert D[0]["flags"] & 2 == 0
    finally:
        eng.close()
