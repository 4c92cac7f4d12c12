"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
entry point that include/pepo.h declares, and its host-side sizing logic
accepts / rejects configurations (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2606_30985_gb300 as pkg
from paper_2606_30985_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return pkg.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pepo.h")).read()
    return sorted(set(re.findall(r"\b(pepo_[a-z_]+)\s*\(", text)))


def test_header_declares_the_method_entry_points():
    names = declared_symbols()
    for required in ("pepo_init", "pepo_trotter_step", "pepo_bp_converge", "pepo_correlator"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(declared_symbols()) == sorted(pkg.EXPORTS)


def test_config_default_matches_paper_defaults(lib):
    c = pkg._Config()
    lib.pepo_config_default(ctypes.byref(c))
    assert c.eps_cut == 1e-11 and c.bp_tol == 1e-5 and c.bp_max_sweeps == 100
    assert c.qr_n_thresh == 150 and c.qr_ratio_thresh == 150.0
    assert c.gates == 0 and c.trotter_order == 1


def test_required_bytes_valid_and_invalid(lib):
    small = pkg.required_bytes(pkg.Config(Lx=3, Ly=3, chi_max=8, precision="fp64"))
    assert small > 0
    # larger chi and FP64 storage need more memory
    assert pkg.required_bytes(pkg.Config(Lx=3, Ly=3, chi_max=16, precision="fp64")) > small
    assert pkg.required_bytes(pkg.Config(Lx=1, Ly=1)) == 0           # one site
    assert pkg.required_bytes(pkg.Config(Lx=3, Ly=3, chi_max=200)) == 0  # beyond the kernel bound
    assert pkg.required_bytes(pkg.Config(Lx=3, Ly=3, obs=(5, 0))) == 0
    assert pkg.required_bytes(pkg.Config(Lx=3, Ly=3, order=3)) == 0
    # mixed precisions in one context are rejected
    assert pkg.required_bytes([pkg.Config(precision="fp32"), pkg.Config(precision="fp64")]) == 0


def test_required_bytes_follow_the_memory_model(lib):
    # Eq. 15: the site tensors alone are (4 chi^2 + 2 (k+l-4) chi^3 + (k-2)(l-2) chi^4) * 4 * 4 B
    k = l = 10
    chi = 100
    m_psi = (4 * chi ** 2 + 2 * (k + l - 4) * chi ** 3 + (k - 2) * (l - 2) * chi ** 4) * 4 * 4
    need = pkg.required_bytes(pkg.Config(Lx=k, Ly=l, chi_max=chi))
    assert m_psi < need < 180e9


@pytest.mark.parametrize("field,value", [
    ("bp_alpha", 0.0), ("bp_alpha", 1.5), ("bp_tol", 0.0), ("bp_max_sweeps", 0),
    ("eps_cut", -1e-3), ("chi_max", 0), ("h", float("nan")), ("dt", float("inf")),
    ("inflight_sites", -1)])
def test_required_bytes_rejects_each_invalid_field(lib, field, value):
    assert pkg.required_bytes(pkg.Config(Lx=3, Ly=3, chi_max=8)) > 0
    cfg = pkg.Config(Lx=3, Ly=3, chi_max=8)
    setattr(cfg, field, value)
    assert pkg.required_bytes(cfg) == 0


def test_required_bytes_rejects_invalid_raw_fields(lib):
    def raw(**kw):
        c = pkg.Config(Lx=3, Ly=3, chi_max=8).to_c()
        for k, v in kw.items():
            setattr(c, k, v)
        arr = (pkg._Config * 1)(c)
        return int(lib.pepo_required_bytes(arr, 1))
    assert raw() > 0
    assert raw(obs_pauli=0) == 0 and raw(obs_pauli=4) == 0
    assert raw(gates=2) == 0 and raw(prec=4) == 0 and raw(prec=-1) == 0
    assert raw(prec=2) > 0 and raw(prec=3) == 0          # BF16X3 is refused, not aliased
    assert raw(Lx=65, Ly=65) == 0                      # more than 4096 sites
    assert raw(Lx=2, Ly=1, obs_x=1, obs_y=0) > 0       # a two-site chain is a valid grid


def test_every_context_call_refuses_a_null_context(lib):
    # host-side guards: no CUDA call is reached
    null = None
    I, D = ctypes.c_int, ctypes.c_double
    assert lib.pepo_trotter_step(null, 1) == 1
    assert lib.pepo_trotter_colour(null, 0) == 1
    assert lib.pepo_set_wait_limit(null, 1.0) == 1
    assert lib.pepo_save_state_host(null, 0, None, 0, None) == 1
    assert lib.pepo_load_state_host(null, 0, None, 0, 0) == 1
    assert lib.pepo_bp_converge(null, None, None) == 1
    assert lib.pepo_correlator(null, None, None) == 1
    assert lib.pepo_get_spectrum(null, 0, 0, (D * 4)(), ctypes.byref(I())) == 1
    assert lib.pepo_set_site(null, 0, 0, None, 0, 0) == 1
    assert lib.pepo_save_state(null, 0, None, 0) == 1
    assert lib.pepo_load_state(null, 0, None, 0) == 1
    assert lib.pepo_set_timing(null, 1) == 1 and lib.pepo_reset_timing(null) == 1
    assert lib.pepo_set_tuning(null, ctypes.byref(pkg._Tuning())) == 1
    assert lib.pepo_get_tuning(null, ctypes.byref(pkg._Tuning())) == 1
    assert lib.pepo_set_warmstart_weights(null, None, 0) == 1
    assert lib.pepo_set_bp_params(null, 0, 0.5, 1e-5, 100) == 1
    assert lib.pepo_get_messages(null, 0, None) == 1 and lib.pepo_set_messages(null, 0, None) == 1
    assert lib.pepo_state_bytes(null, 0) == 0 and lib.pepo_num_bonds(null, 0) == 0
    assert lib.pepo_launch_count(null) == 0
    assert lib.pepo_last_error(null)          # a message, not a null pointer
    lib.pepo_destroy(null)                    # a no-op


def test_init_refusals_happen_before_any_device_access(lib):
    cfg = pkg.Config(Lx=3, Ly=3, chi_max=8).to_c()
    arr = (pkg._Config * 1)(cfg)
    need = int(lib.pepo_required_bytes(arr, 1))
    fake = ctypes.c_void_p(1 << 20)              # aligned, never dereferenced on these paths
    out = ctypes.c_void_p(123)

    def init(cfgs=arr, n=1, arena=fake, nbytes=need, outp=True):
        out.value = 123
        return lib.pepo_init(cfgs, n, arena, nbytes, None, ctypes.byref(out) if outp else None)

    assert init(nbytes=need - 1) == 2 and not out.value          # PEPO_E_OOM, *out = NULL
    assert init(nbytes=0) == 2 and not out.value
    assert init(arena=ctypes.c_void_p((1 << 20) + 8)) == 1 and not out.value   # misaligned
    assert init(arena=None) == 1 and init(n=0) == 1 and init(cfgs=None) == 1
    assert init(outp=False) == 1
    bad = pkg.Config(Lx=3, Ly=3, chi_max=8, bp_alpha=0.0).to_c()
    assert init(cfgs=(pkg._Config * 1)(bad)) == 1 and not out.value


def test_mlp_entry_points_refuse_bad_arguments_on_the_host(lib):
    n = int(lib.pepo_mlp_num_params())
    assert n > 0
    assert lib.pepo_mlp_required_bytes(0) == 0
    need = int(lib.pepo_mlp_required_bytes(64))
    assert need > 4 * n
    params = (ctypes.c_float * n)()
    out = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(1 << 20)
    assert lib.pepo_mlp_init(fake, need - 1, 64, params, None, ctypes.byref(out)) == 2 and not out.value
    assert lib.pepo_mlp_init(ctypes.c_void_p((1 << 20) + 4), need, 64, params, None, ctypes.byref(out)) == 1
    assert lib.pepo_mlp_init(fake, need, 0, params, None, ctypes.byref(out)) == 1
    assert lib.pepo_mlp_init(fake, need, 64, None, None, ctypes.byref(out)) == 1
    assert lib.pepo_mlp_forward(None, fake, 1, fake) == 1
    assert lib.pepo_mlp_gradient(None, fake, fake, 1, None, None) == 1
    assert lib.pepo_mlp_adam_step(None, 1e-3) == 1
    assert lib.pepo_ws_rows(None, 0) == -1
    lib.pepo_mlp_destroy(None)
