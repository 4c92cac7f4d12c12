"""GB300-native Heisenberg-picture PEPO evolution of the 2D transverse-field Ising model.

Thin ctypes binding of ``libpepo.so`` (C ABI in ``include/pepo.h``).  Every step
of the method runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch supplies the device arena (one uint8 tensor) and the stream.
There is no CPU fallback: if the library or a CUDA device is missing, the
constructor raises.
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpepo.so")

GATES = {"ZZ_X": 0, "XX_Z": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3}
PAULI = {"X": 1, "Y": 2, "Z": 3}
STATUS = {0: "ok", 1: "invalid argument", 2: "arena too small", 3: "CUDA error",
          4: "numeric failure", 5: "call out of order"}


class PepoError(RuntimeError):
    pass


class _Config(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int),
                ("J", ctypes.c_double), ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("trotter_order", ctypes.c_int),
                ("obs_x", ctypes.c_int), ("obs_y", ctypes.c_int), ("obs_pauli", ctypes.c_int),
                ("chi_max", ctypes.c_int), ("eps_cut", ctypes.c_double),
                ("bp_alpha", ctypes.c_double), ("bp_tol", ctypes.c_double),
                ("bp_max_sweeps", ctypes.c_int),
                ("qr_n_thresh", ctypes.c_int), ("qr_ratio_thresh", ctypes.c_double),
                ("pinv_rel", ctypes.c_double),
                ("gates", ctypes.c_int), ("prec", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("inflight_sites", ctypes.c_int)]


class _Diag(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double), ("C_proj", ctypes.c_double), ("log_norm", ctypes.c_double),
                ("gate_err", ctypes.c_double), ("bp_sweeps", ctypes.c_int),
                ("bp_delta", ctypes.c_double), ("bp1_sweeps", ctypes.c_int),
                ("bp1_delta", ctypes.c_double), ("entropy_frac_max", ctypes.c_double),
                ("trap_type1", ctypes.c_int), ("trap_type2", ctypes.c_int),
                ("norm_exploded", ctypes.c_int), ("flags", ctypes.c_int), ("steps", ctypes.c_int),
                ("core_sweeps32_max", ctypes.c_int), ("core_sweeps64_max", ctypes.c_int),
                ("c_drop", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("gram_leg_splits", ctypes.c_int), ("gram_rows_splits", ctypes.c_int)]


EXPORTS = ["pepo_config_default", "pepo_required_bytes", "pepo_init", "pepo_trotter_step", "pepo_trotter_colour",
           "pepo_bp_converge", "pepo_correlator", "pepo_get_spectrum", "pepo_get_site",
           "pepo_set_state", "pepo_set_bonds", "pepo_set_site", "pepo_set_site_static", "pepo_state_bytes", "pepo_save_state", "pepo_load_state",
           "pepo_get_message", "pepo_num_bonds", "pepo_set_timing", "pepo_set_tuning", "pepo_get_tuning",
           "pepo_timing_classes", "pepo_timing_class_name", "pepo_get_timing", "pepo_reset_timing",
           "pepo_launch_count", "pepo_last_error", "pepo_destroy",
           "pepo_mlp_num_params", "pepo_mlp_required_bytes", "pepo_mlp_init", "pepo_mlp_get_params",
           "pepo_mlp_forward", "pepo_mlp_gradient", "pepo_mlp_adam_step", "pepo_mlp_destroy",
           "pepo_ws_rows", "pepo_ws_features", "pepo_ws_targets", "pepo_ws_apply", "pepo_set_warmstart_weights",
           "pepo_c_drop", "pepo_set_bp_params", "pepo_get_messages", "pepo_set_messages",
           "pepo_set_wait_limit", "pepo_save_state_host", "pepo_load_state_host", "pepo_pauli_weights",
           "pepo_qr_branch_counts"]

_lib = None

# learned warm start: feature count, hidden width, default blend of the
# prediction with the diag(lambda) start (best of {1, 0.5, 0.25} in the 6x6 study)
WS_FEATURES = 12
WS_WIDTH = 256
WS_GAMMA = 0.25


def _device_tensor(t, dtype, min_numel, what):
    """Raise PepoError unless t is a contiguous CUDA tensor of `dtype` with at
    least min_numel elements (the library receives only its raw pointer)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise PepoError("%s: expected a torch tensor, got %s" % (what, type(t).__name__))
    if not t.is_cuda:
        raise PepoError("%s: the tensor must live on the GPU" % what)
    if t.dtype != dtype:
        raise PepoError("%s: expected dtype %s, got %s" % (what, dtype, t.dtype))
    if not t.is_contiguous():
        raise PepoError("%s: the tensor must be contiguous" % what)
    if t.numel() < min_numel:
        raise PepoError("%s: %d elements, at least %d needed" % (what, t.numel(), min_numel))
    return t


def load_library(path=LIB_PATH):
    """Load libpepo.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PepoError("libpepo.so not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    CP = ctypes.POINTER(_Config)
    lib.pepo_config_default.argtypes = [CP]
    lib.pepo_config_default.restype = None
    lib.pepo_c_drop.argtypes = [ctypes.c_double] * 4
    lib.pepo_c_drop.restype = ctypes.c_int
    lib.pepo_set_bp_params.argtypes = [P, I, D, D, I]
    lib.pepo_get_messages.argtypes = [P, I, ctypes.POINTER(D)]
    lib.pepo_set_messages.argtypes = [P, I, ctypes.POINTER(D)]
    lib.pepo_required_bytes.argtypes = [CP, I]
    lib.pepo_required_bytes.restype = S
    lib.pepo_init.argtypes = [CP, I, P, S, P, ctypes.POINTER(P)]
    lib.pepo_init.restype = I
    lib.pepo_trotter_step.argtypes = [P, I]
    lib.pepo_trotter_step.restype = I
    lib.pepo_trotter_colour.argtypes = [P, I]
    lib.pepo_trotter_colour.restype = I
    lib.pepo_bp_converge.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.pepo_bp_converge.restype = I
    lib.pepo_correlator.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(_Diag)]
    lib.pepo_correlator.restype = I
    lib.pepo_get_spectrum.argtypes = [P, I, I, ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.pepo_get_spectrum.restype = I
    lib.pepo_get_site.argtypes = [P, I, I, ctypes.POINTER(D), S, ctypes.POINTER(I)]
    lib.pepo_get_site.restype = I
    lib.pepo_set_state.argtypes = [P, I, ctypes.POINTER(D), S, ctypes.POINTER(I), ctypes.POINTER(D),
                                   ctypes.POINTER(D)]
    lib.pepo_set_state.restype = I
    lib.pepo_set_bonds.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.pepo_set_bonds.restype = I
    lib.pepo_set_site.argtypes = [P, I, I, P, I, S]
    lib.pepo_set_site.restype = I
    lib.pepo_set_site_static.argtypes = [P, I, I, P, I, S]
    lib.pepo_set_site_static.restype = I
    lib.pepo_state_bytes.argtypes = [P, I]
    lib.pepo_state_bytes.restype = S
    lib.pepo_save_state.argtypes = [P, I, P, S]
    lib.pepo_save_state.restype = I
    lib.pepo_load_state.argtypes = [P, I, P, S]
    lib.pepo_load_state.restype = I
    lib.pepo_save_state_host.argtypes = [P, I, P, S, ctypes.POINTER(I)]
    lib.pepo_save_state_host.restype = I
    lib.pepo_load_state_host.argtypes = [P, I, P, S, I]
    lib.pepo_load_state_host.restype = I
    F = ctypes.c_float
    FP = ctypes.POINTER(ctypes.c_float)
    lib.pepo_mlp_num_params.argtypes = []
    lib.pepo_mlp_num_params.restype = ctypes.c_longlong
    lib.pepo_mlp_required_bytes.argtypes = [I]
    lib.pepo_mlp_required_bytes.restype = S
    lib.pepo_mlp_init.argtypes = [P, S, I, FP, P, ctypes.POINTER(P)]
    lib.pepo_mlp_init.restype = I
    lib.pepo_mlp_get_params.argtypes = [P, FP]
    lib.pepo_mlp_get_params.restype = I
    lib.pepo_mlp_forward.argtypes = [P, P, I, P]
    lib.pepo_mlp_forward.restype = I
    lib.pepo_mlp_gradient.argtypes = [P, P, P, I, FP, FP]
    lib.pepo_mlp_gradient.restype = I
    lib.pepo_mlp_adam_step.argtypes = [P, F]
    lib.pepo_mlp_adam_step.restype = I
    lib.pepo_mlp_destroy.argtypes = [P]
    lib.pepo_mlp_destroy.restype = None
    lib.pepo_ws_rows.argtypes = [P, I]
    lib.pepo_ws_rows.restype = I
    lib.pepo_ws_features.argtypes = [P, I, P, I]
    lib.pepo_ws_features.restype = I
    lib.pepo_ws_targets.argtypes = [P, I, P, I]
    lib.pepo_ws_targets.restype = I
    lib.pepo_ws_apply.argtypes = [P, I, P, F]
    lib.pepo_ws_apply.restype = I
    lib.pepo_set_warmstart_weights.argtypes = [P, P, S]
    lib.pepo_set_warmstart_weights.restype = I
    lib.pepo_pauli_weights.argtypes = [P, I, ctypes.POINTER(D)]
    lib.pepo_pauli_weights.restype = I
    lib.pepo_get_message.argtypes = [P, I, I, I, ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.pepo_get_message.restype = I
    lib.pepo_num_bonds.argtypes = [P, I]
    lib.pepo_num_bonds.restype = I
    lib.pepo_set_timing.argtypes = [P, I]
    lib.pepo_set_timing.restype = I
    lib.pepo_set_wait_limit.argtypes = [P, D]
    lib.pepo_set_wait_limit.restype = I
    lib.pepo_set_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    lib.pepo_set_tuning.restype = I
    lib.pepo_get_tuning.argtypes = [P, ctypes.POINTER(_Tuning)]
    lib.pepo_get_tuning.restype = I
    lib.pepo_timing_classes.argtypes = []
    lib.pepo_timing_classes.restype = I
    lib.pepo_timing_class_name.argtypes = [I]
    lib.pepo_timing_class_name.restype = ctypes.c_char_p
    lib.pepo_get_timing.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                    ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.pepo_get_timing.restype = I
    lib.pepo_reset_timing.argtypes = [P]
    lib.pepo_reset_timing.restype = I
    lib.pepo_qr_branch_counts.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), I]
    lib.pepo_qr_branch_counts.restype = I
    lib.pepo_launch_count.argtypes = [P]
    lib.pepo_launch_count.restype = ctypes.c_longlong
    lib.pepo_last_error.argtypes = [P]
    lib.pepo_last_error.restype = ctypes.c_char_p
    lib.pepo_destroy.argtypes = [P]
    lib.pepo_destroy.restype = None
    _lib = lib
    return lib


@dataclass
class Config:
    """One instance of the method (mirrors pepo_config; defaults of Sec. 6)."""
    Lx: int = 3
    Ly: int = 3
    J: float = 1.0
    h: float = 1.0
    dt: float = 0.05
    order: int = 1
    obs: tuple = None
    obs_pauli: str = "Z"
    chi_max: int = 8
    eps_cut: float = 1e-11
    bp_alpha: float = 0.5
    bp_tol: float = 1e-5
    bp_max_sweeps: int = 100
    qr_n_thresh: int = 150
    qr_ratio_thresh: float = 150.0
    pinv_rel: float = 1e-12
    gateset: str = "ZZ_X"
    precision: str = "fp32"
    inflight_sites: int = 0
    warm_start: int = 0

    def to_c(self):
        c = _Config()
        obs = self.obs if self.obs is not None else ((self.Lx - 1) // 2, (self.Ly - 1) // 2)
        c.Lx, c.Ly = self.Lx, self.Ly
        c.J, c.h, c.dt = self.J, self.h, self.dt
        c.trotter_order = self.order
        c.obs_x, c.obs_y = obs
        c.obs_pauli = PAULI[self.obs_pauli]
        c.chi_max = self.chi_max
        c.eps_cut = self.eps_cut
        c.bp_alpha, c.bp_tol, c.bp_max_sweeps = self.bp_alpha, self.bp_tol, self.bp_max_sweeps
        c.qr_n_thresh, c.qr_ratio_thresh = self.qr_n_thresh, self.qr_ratio_thresh
        c.pinv_rel = self.pinv_rel
        c.gates = GATES[self.gateset]
        c.prec = PRECISIONS[self.precision]
        c.warm_start = int(self.warm_start)
        c.inflight_sites = self.inflight_sites
        return c


def _cfg_array(cfgs):
    arr = (_Config * len(cfgs))()
    for i, c in enumerate(cfgs):
        arr[i] = c.to_c()
    return arr


def required_bytes(cfgs):
    """Device bytes pepo_init needs (host-only computation; 0 for an invalid config)."""
    if isinstance(cfgs, Config):
        cfgs = [cfgs]
    lib = load_library()
    return int(lib.pepo_required_bytes(_cfg_array(cfgs), len(cfgs)))


def diag_to_dict(d):
    return {name: getattr(d, name) for name, _ in _Diag._fields_}


class Engine:
    """A context of one or more instances living in one device arena."""

    def __init__(self, cfgs, device="cuda:0", tuning="cache"):
        """tuning: "cache" applies the launch shapes that the autotuner cached
        for the nearest class of (chi_max, precision) (autotune.lookup), None
        keeps the built-in shapes, a dict sets them (Engine.set_tuning)."""
        import torch
        if isinstance(cfgs, Config):
            cfgs = [cfgs]
        self.cfgs = list(cfgs)
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise PepoError("a CUDA device is required (no CPU fallback)")
        self.device = torch.device(device)
        arr = _cfg_array(self.cfgs)
        nbytes = int(self.lib.pepo_required_bytes(arr, len(self.cfgs)))
        if nbytes == 0:
            raise PepoError("invalid configuration")
        with torch.cuda.device(self.device):
            self.arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
        self.arena_bytes = nbytes
        ctx = ctypes.c_void_p()
        st = self.lib.pepo_init(arr, len(self.cfgs), ctypes.c_void_p(self.arena.data_ptr()),
                                nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if st != 0:
            raise PepoError("pepo_init failed: %s" % STATUS.get(st, st))
        self.ctx = ctx
        self._bp = [(c.bp_alpha, c.bp_tol, c.bp_max_sweeps) for c in self.cfgs]
        if tuning == "cache":
            from . import autotune
            tuning = autotune.lookup(max(c.chi_max for c in self.cfgs), self.cfgs[0].precision)
        if tuning:
            self.set_tuning(**tuning)

    # -- helpers
    def _check(self, st, what):
        if st != 0:
            msg = self.lib.pepo_last_error(self.ctx).decode()
            raise PepoError("%s failed (%s): %s" % (what, STATUS.get(st, st), msg))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pepo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_inst(self):
        return len(self.cfgs)

    def launches(self):
        return int(self.lib.pepo_launch_count(self.ctx))

    def qr_branch_counts(self, reset=True):
        """Sites factored by each hybrid-QR branch (Sec. 4.2) since the last
        reset: householder (branch rule), cholesky, cholesky_fallback (a Gram
        pivot kept too small a share of its column's diagonal)."""
        out = (ctypes.c_longlong * 3)()
        self._check(self.lib.pepo_qr_branch_counts(self.ctx, out, 1 if reset else 0), "pepo_qr_branch_counts")
        return dict(householder=int(out[0]), cholesky=int(out[1]), cholesky_fallback=int(out[2]))

    def set_tuning(self, gram_leg_splits=0, gram_rows_splits=0):
        """Launch shapes (pepo_set_tuning): K splits of the free-leg and the
        Cholesky-QR Grams, 0 = default."""
        t = _Tuning(int(gram_leg_splits), int(gram_rows_splits))
        self._check(self.lib.pepo_set_tuning(self.ctx, ctypes.byref(t)), "pepo_set_tuning")

    def set_wait_limit(self, seconds):
        """Limit of every tensor-core pipeline wait (pepo_set_wait_limit)."""
        self._check(self.lib.pepo_set_wait_limit(self.ctx, float(seconds)), "pepo_set_wait_limit")

    def get_tuning(self):
        t = _Tuning()
        self._check(self.lib.pepo_get_tuning(self.ctx, ctypes.byref(t)), "pepo_get_tuning")
        return {"gram_leg_splits": t.gram_leg_splits, "gram_rows_splits": t.gram_rows_splits}

    def set_timing(self, on=True):
        self._check(self.lib.pepo_set_timing(self.ctx, 1 if on else 0), "pepo_set_timing")

    def reset_timing(self):
        self._check(self.lib.pepo_reset_timing(self.ctx), "pepo_reset_timing")

    def timing(self):
        """{class: dict(launches, ms, bytes, flops)} since the last reset."""
        out = {}
        for k in range(self.lib.pepo_timing_classes()):
            n = ctypes.c_longlong()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.pepo_get_timing(self.ctx, k, ctypes.byref(n), ctypes.byref(ms),
                                                 ctypes.byref(by), ctypes.byref(fl)), "pepo_get_timing")
            out[self.lib.pepo_timing_class_name(k).decode()] = dict(
                launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)
        return out

    # -- the four entry points of the method
    def trotter_step(self, n=1):
        self._check(self.lib.pepo_trotter_step(self.ctx, n), "pepo_trotter_step")

    def trotter_colour(self, colour):
        """Bond gates of one colour class of the current step (colours in the
        order 0..3; the four together equal trotter_step(1))."""
        self._check(self.lib.pepo_trotter_colour(self.ctx, int(colour)), "pepo_trotter_colour")

    def bp_converge(self):
        sw = (ctypes.c_int * self.n_inst)()
        de = (ctypes.c_double * self.n_inst)()
        self._check(self.lib.pepo_bp_converge(self.ctx, sw, de), "pepo_bp_converge")
        return list(sw), list(de)

    def correlator(self):
        C = (ctypes.c_double * self.n_inst)()
        D = (_Diag * self.n_inst)()
        self._check(self.lib.pepo_correlator(self.ctx, C, D), "pepo_correlator")
        return list(C), [diag_to_dict(d) for d in D]

    # -- BP settings and message snapshots (trap remediation)
    def set_bp_params(self, alpha, tol=None, max_sweeps=None, inst=-1):
        """Damping / tolerance / sweep budget of instance inst (-1: all) for the
        following BP runs (pepo_set_bp_params); None keeps a value."""
        targets = range(self.n_inst) if inst < 0 else [inst]
        for i in targets:
            a0, t0, m0 = self.bp_params(i)
            t = t0 if tol is None else tol
            m = m0 if max_sweeps is None else max_sweeps
            self._check(self.lib.pepo_set_bp_params(self.ctx, i, float(alpha), float(t), int(m)),
                        "pepo_set_bp_params")
            self._bp[i] = (float(alpha), float(t), int(m))

    def bp_params(self, inst=0):
        """(alpha, tol, max_sweeps) in force for instance inst."""
        return self._bp[inst]

    def get_messages(self, inst=0):
        """All double-layer messages as stored (2 * num_bonds x chi_max x chi_max)."""
        cm = self.cfgs[inst].chi_max
        out = np.zeros((2 * self.num_bonds(inst), cm, cm))
        self._check(self.lib.pepo_get_messages(self.ctx, inst, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "pepo_get_messages")
        return out

    def set_messages(self, msgs, inst=0):
        cm = self.cfgs[inst].chi_max
        m = np.ascontiguousarray(np.asarray(msgs, dtype=np.float64))
        if m.size != 2 * self.num_bonds(inst) * cm * cm:
            raise PepoError("set_messages: expected %d values, got %d" % (2 * self.num_bonds(inst) * cm * cm, m.size))
        self._check(self.lib.pepo_set_messages(self.ctx, inst, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "pepo_set_messages")

    def measure_remediated(self, alphas=None, inst=0):
        """BP + correlator with the Sec. 6.3 trap remediation (remediation.measure)."""
        from . import remediation
        return remediation.measure(self, inst=inst, alphas=alphas or remediation.ALPHAS)

    # -- state access
    def num_bonds(self, inst=0):
        return int(self.lib.pepo_num_bonds(self.ctx, inst))

    def spectrum(self, inst, bond):
        cm = self.cfgs[inst].chi_max
        lam = (ctypes.c_double * cm)()
        chi = ctypes.c_int()
        self._check(self.lib.pepo_get_spectrum(self.ctx, inst, bond, lam, ctypes.byref(chi)),
                    "pepo_get_spectrum")
        return np.array(lam[: chi.value])

    def site(self, inst, v):
        cm = self.cfgs[inst].chi_max
        cap = 4 * cm ** 4
        buf = np.zeros(cap)
        dims = (ctypes.c_int * 4)()
        self._check(self.lib.pepo_get_site(self.ctx, inst, v, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           cap, dims), "pepo_get_site")
        d = [x for x in dims if x > 0]
        n = 4 * int(np.prod(d)) if d else 4
        return buf[:n].reshape(tuple(d) + (4,)), list(dims)

    def pauli_weights(self, inst=0):
        """[Ly, Lx, 4] Pauli weights (I, X, Y, Z) per site from the last
        correlator call (pepo_pauli_weights); rows sum to 1."""
        c = self.cfgs[inst]
        out = np.zeros(4 * c.Lx * c.Ly)
        self._check(self.lib.pepo_pauli_weights(self.ctx, inst, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "pepo_pauli_weights")
        return out.reshape(c.Ly, c.Lx, 4)

    def spatial(self, inst=0):
        """Operator spreading of the last correlator call (Sec. 6.4, Appendix
        A.3): n(r) = 1 - I-weight per site, the mean Manhattan radius R_L1 and
        the RMS Euclidean radius R_L2 from the observable site with weights
        p(r) = n(r) / sum n, and S_frac = -sum p ln p / ln(number of sites)."""
        w = self.pauli_weights(inst)
        n = 1.0 - w[..., 0]
        return spatial_observables(n, self.cfgs[inst])

    def message(self, inst, bond, direction):
        cm = self.cfgs[inst].chi_max
        buf = np.zeros(cm * cm)
        chi = ctypes.c_int()
        self._check(self.lib.pepo_get_message(self.ctx, inst, bond, direction,
                                              buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              ctypes.byref(chi)), "pepo_get_message")
        k = chi.value
        return buf[: k * k].reshape(k, k)

    def set_state(self, inst, sites, chi, lam, msgs):
        """sites: list of arrays in canonical layout; chi: per bond; lam: [nb, chi_max];
        msgs: [nb, 2, chi_max, chi_max]."""
        flat = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.float64).ravel() for s in sites]))
        chi = np.ascontiguousarray(np.asarray(chi, dtype=np.int32))
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
        msgs = np.ascontiguousarray(np.asarray(msgs, dtype=np.float64))
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.pepo_set_state(self.ctx, inst, flat.ctypes.data_as(dp), flat.size,
                                            chi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                            lam.ctypes.data_as(dp), msgs.ctypes.data_as(dp)),
                    "pepo_set_state")

    def set_bonds(self, inst, chi, lam, msgs):
        chi = np.ascontiguousarray(np.asarray(chi, dtype=np.int32))
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
        msgs = np.ascontiguousarray(np.asarray(msgs, dtype=np.float64))
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.pepo_set_bonds(self.ctx, inst, chi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                            lam.ctypes.data_as(dp), msgs.ctypes.data_as(dp)),
                    "pepo_set_bonds")

    def set_site(self, inst, v, tensor):
        """tensor: canonical layout [legs..., 4], float32 or float64."""
        t = np.ascontiguousarray(tensor)
        if t.dtype == np.float32:
            dt = 0
        else:
            t = np.ascontiguousarray(t, dtype=np.float64)
            dt = 1
        self._check(self.lib.pepo_set_site(self.ctx, inst, v, ctypes.c_void_p(t.ctypes.data), dt, t.size),
                    "pepo_set_site")

    def set_site_static(self, inst, v, tensor):
        """As set_site, through the library's fixed device staging buffer (no
        allocation); tensor must already have the storage dtype."""
        t = np.ascontiguousarray(tensor)
        if t.dtype not in (np.float32, np.float64):
            raise PepoError("set_site_static: float32 or float64 data required, got %s" % t.dtype)
        dt = 0 if t.dtype == np.float32 else 1
        self._check(self.lib.pepo_set_site_static(self.ctx, inst, v, ctypes.c_void_p(t.ctypes.data), dt,
                                                  t.size), "pepo_set_site_static")

    # -- state snapshot
    def state_bytes(self, inst=0):
        return int(self.lib.pepo_state_bytes(self.ctx, inst))

    def save_state(self, buf, inst=0):
        """Copy the instance's state into the device tensor `buf` (uint8)."""
        import torch
        _device_tensor(buf, torch.uint8, self.state_bytes(inst), "save_state")
        self._check(self.lib.pepo_save_state(self.ctx, inst, ctypes.c_void_p(buf.data_ptr()), buf.numel()),
                    "pepo_save_state")

    def load_state(self, buf, inst=0):
        import torch
        _device_tensor(buf, torch.uint8, self.state_bytes(inst), "load_state")
        self._check(self.lib.pepo_load_state(self.ctx, inst, ctypes.c_void_p(buf.data_ptr()), buf.numel()),
                    "pepo_load_state")

    # -- checkpoint / restart through host memory
    def checkpoint(self, path, inst=0):
        """Write instance inst's state (pepo_save_state_host) and its step
        count to `path` (numpy .npz)."""
        buf = np.empty(self.state_bytes(inst), dtype=np.uint8)
        steps = ctypes.c_int()
        self._check(self.lib.pepo_save_state_host(self.ctx, inst, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                                  ctypes.byref(steps)), "pepo_save_state_host")
        c = self.cfgs[inst]
        np.savez(path, state=buf, steps=steps.value,
                 config=np.array(repr(sorted(vars(c).items()))))
        return steps.value

    def restore(self, path, inst=0):
        """Restart instance inst from a checkpoint written by checkpoint()
        for the same configuration."""
        with np.load(path) as z:
            if str(z["config"]) != repr(sorted(vars(self.cfgs[inst]).items())):
                raise PepoError("restore: the checkpoint was written for another configuration")
            buf = np.ascontiguousarray(z["state"])
            steps = int(z["steps"])
        if buf.size != self.state_bytes(inst):
            raise PepoError("restore: %d bytes in the checkpoint, %d expected" % (buf.size, self.state_bytes(inst)))
        self._check(self.lib.pepo_load_state_host(self.ctx, inst, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                                  steps), "pepo_load_state_host")
        return steps

    # -- learned warm start
    def ws_rows(self, inst=0):
        r = int(self.lib.pepo_ws_rows(self.ctx, inst))
        if r < 0:
            raise PepoError("pepo_ws_rows failed")
        return r

    def ws_features(self, inst=0, out=None):
        """Feature rows (torch float32 [rows, 12] on the device)."""
        import torch
        r = self.ws_rows(inst)
        X = out if out is not None else torch.empty((r, WS_FEATURES), dtype=torch.float32, device=self.device)
        _device_tensor(X, torch.float32, 0, "ws_features")
        if X.dim() != 2 or X.shape[1] != WS_FEATURES:
            raise PepoError("ws_features: out must be [rows, %d]" % WS_FEATURES)
        self._check(self.lib.pepo_ws_features(self.ctx, inst, ctypes.c_void_p(X.data_ptr()), X.shape[0]),
                    "pepo_ws_features")
        return X

    def ws_targets(self, inst=0, out=None):
        """log diag of the current messages (torch float32 [rows])."""
        import torch
        r = self.ws_rows(inst)
        t = out if out is not None else torch.empty((r,), dtype=torch.float32, device=self.device)
        _device_tensor(t, torch.float32, 0, "ws_targets")
        self._check(self.lib.pepo_ws_targets(self.ctx, inst, ctypes.c_void_p(t.data_ptr()), t.shape[0]),
                    "pepo_ws_targets")
        return t

    def ws_apply(self, y, inst=0, gamma=1.0):
        """Messages <- diag((1-gamma) d/sum d + gamma exp(y)/sum exp(y)) per directed bond."""
        import torch
        _device_tensor(y, torch.float32, self.ws_rows(inst), "ws_apply")
        if not 0.0 <= gamma <= 1.0:
            raise PepoError("ws_apply: gamma must lie in [0, 1]")
        self._check(self.lib.pepo_ws_apply(self.ctx, inst, ctypes.c_void_p(y.data_ptr()), ctypes.c_float(gamma)),
                    "pepo_ws_apply")

    def set_warmstart_weights(self, params):
        """Install the warm-start network for pepo_bp_converge (instances
        created with warm_start=1): params is a device float32 tensor of
        pepo_mlp_num_params entries (e.g. a trained Mlp's parameters)."""
        import torch
        n = int(self.lib.pepo_mlp_num_params())
        _device_tensor(params, torch.float32, n, "set_warmstart_weights")
        self._check(self.lib.pepo_set_warmstart_weights(self.ctx, ctypes.c_void_p(params.data_ptr()), 4 * n),
                    "pepo_set_warmstart_weights")

    def ws_warm_start(self, mlp, inst=0, gamma=WS_GAMMA):
        """Predict the converged message diagonals with `mlp` and install them
        (blended with the current diag(lambda) start by gamma)."""
        X = self.ws_features(inst)
        y = mlp.forward(X)
        self.ws_apply(y, inst, gamma)
        return X.shape[0]

    def run(self, nsteps, measure_every=1):
        """Evolve nsteps, measuring C(t) (BP + correlator) every `measure_every` steps."""
        out = []
        pick = (lambda D: D[0]) if self.n_inst == 1 else (lambda D: D)
        self.bp_converge()
        C, D = self.correlator()
        out.append(pick(D))
        for s in range(1, nsteps + 1):
            self.trotter_step(1)
            if s % measure_every == 0 or s == nsteps:
                self.bp_converge()
                C, D = self.correlator()
                out.append(pick(D))
        return out



class Mlp:
    """The warm-start network (device buffer owned here, kernels in libpepo)."""

    def __init__(self, params, max_rows, device="cuda:0"):
        import torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise PepoError("a CUDA device is required (no CPU fallback)")
        self.device = torch.device(device)
        self.n = int(self.lib.pepo_mlp_num_params())
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != self.n:
            raise PepoError("expected %d parameters, got %d" % (self.n, p.size))
        nbytes = int(self.lib.pepo_mlp_required_bytes(max_rows))
        with torch.cuda.device(self.device):
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
        self.max_rows = max_rows
        h = ctypes.c_void_p()
        st = self.lib.pepo_mlp_init(ctypes.c_void_p(self.buf.data_ptr()), nbytes, max_rows,
                                    p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise PepoError("pepo_mlp_init failed: %s" % STATUS.get(st, st))
        self.h = h

    def _ck(self, st, what):
        if st != 0:
            raise PepoError("%s failed (%s)" % (what, STATUS.get(st, st)))

    def params(self):
        out = np.zeros(self.n, dtype=np.float32)
        self._ck(self.lib.pepo_mlp_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                 "pepo_mlp_get_params")
        return out

    def forward(self, X, out=None):
        import torch
        X = X.contiguous()
        y = out if out is not None else torch.empty((X.shape[0],), dtype=torch.float32, device=self.device)
        self._ck(self.lib.pepo_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                           ctypes.c_void_p(y.data_ptr())), "pepo_mlp_forward")
        return y

    def gradient(self, X, t, want_grad=False):
        X = X.contiguous()
        t = t.contiguous()
        loss = ctypes.c_float()
        g = np.zeros(self.n, dtype=np.float32) if want_grad else None
        self._ck(self.lib.pepo_mlp_gradient(self.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                            X.shape[0], ctypes.byref(loss),
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None),
                 "pepo_mlp_gradient")
        return float(loss.value), g

    def adam_step(self, lr):
        self._ck(self.lib.pepo_mlp_adam_step(self.h, ctypes.c_float(lr)), "pepo_mlp_adam_step")

    def close(self):
        if getattr(self, "h", None):
            self.lib.pepo_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spatial_observables(n, cfg):
    """R_L1, R_L2 and S_frac of a non-identity weight map n[y, x] around the
    observable site of cfg (Appendix A.3, Eq. sfrac)."""
    n = np.asarray(n, dtype=np.float64)
    Ly, Lx = n.shape
    ox, oy = cfg.obs if cfg.obs is not None else ((cfg.Lx - 1) // 2, (cfg.Ly - 1) // 2)
    tot = float(np.sum(n))
    yy, xx = np.mgrid[0:Ly, 0:Lx]
    if not tot > 0.0:
        return dict(n=n, R_L1=0.0, R_L2=0.0, S_frac=0.0)
    p = n / tot
    r1 = float(np.sum(p * (np.abs(xx - ox) + np.abs(yy - oy))))
    r2 = float(np.sqrt(np.sum(p * ((xx - ox) ** 2 + (yy - oy) ** 2))))
    nz = p[p > 0.0]
    S = float(-np.sum(nz * np.log(nz)) / np.log(Lx * Ly)) if Lx * Ly > 1 else 0.0
    return dict(n=n, R_L1=r1, R_L2=r2, S_frac=S)


def difference_field(n1, n2):
    """The spatial chi-convergence field of Sec. 6.4: dn(r, t) = n_chi1(r, t) -
    n_chi2(r, t) for two weight maps n[y, x] of the same grid, its largest
    magnitude and, on a square grid, the largest deviation from four-fold
    rotation symmetry about the grid centre (zero for a centred observable
    on an odd grid when both runs are C4-symmetric)."""
    a = np.asarray(n1, dtype=np.float64)
    b = np.asarray(n2, dtype=np.float64)
    if a.shape != b.shape or a.ndim != 2:
        raise PepoError("difference_field: two [Ly, Lx] maps of the same grid expected")
    d = a - b
    out = dict(dn=d, max_abs=float(np.max(np.abs(d))) if d.size else 0.0)
    if d.shape[0] == d.shape[1]:
        out["c4_asym"] = float(max(np.max(np.abs(np.rot90(d, k) - d)) for k in (1, 2, 3)))
    return out


def flat_params(p):
    """Flat parameter vector (library order) from a dict W1, b1, W2, b2, W3, b3."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unflat_params(v):
    F, W = WS_FEATURES, WS_WIDTH
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for k, shape in (("W1", (F, W)), ("b1", (W,)), ("W2", (W, W)), ("b2", (W,)), ("W3", (W, 1)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = v[o:o + n].reshape(shape)
        o += n
    return out
