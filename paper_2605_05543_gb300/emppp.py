"""Python binding of the EM-PP C ABI (``include/emppp.h``): argument marshalling only.

Host arrays are numpy float64 arrays; device arrays are contiguous float64 CUDA tensors (their
pointers are passed with ``is_device_ptr = 1``). Streams are ``torch.cuda.Stream`` objects or raw
``cudaStream_t`` integers. Every computation runs in the library's CUDA kernels; if the library is
missing this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_lib = None

OK, ERR_ARG, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE, ERR_OOM = 0, -1, -2, -3, -4, -5, -6
_STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NUMERIC", -4: "ERR_TIMEOUT", -5: "ERR_STATE",
           -6: "ERR_OOM"}

PRECISION = {"fp64": 0, "mixed": 1}
PROPOSAL = {"bisect": 0, "closed_form": 1, "mlp": 2}
BEXT = {"none": 0, "uniform": 1, "dipole": 2}
# comparison variants of the step: eq:mid, and the self fields at the half-step point
RECONSTRUCTION = {"linear": 0, "midpoint": 1}
FIELD_POINT = {"present": 0, "half_step": 1}


class EmpppError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("proposal", ctypes.c_int32), ("pair_fields", ctypes.c_int32),
                ("source_split", ctypes.c_int32), ("timing", ctypes.c_int32), ("graphs", ctypes.c_int32),
                ("reconstruction", ctypes.c_int32), ("field_point", ctypes.c_int32)]


class Bext(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32), ("b", ctypes.c_double * 3),
                ("m0", ctypes.c_double), ("center", ctypes.c_double * 3)]


class Tuning(ctypes.Structure):
    _fields_ = [("items_per_block", ctypes.c_int32), ("target_order", ctypes.c_int32), ("ms", ctypes.c_double),
                ("targets_per_block", ctypes.c_int32), ("sources_per_sum", ctypes.c_int32),
                ("history_window", ctypes.c_int32)]


class TuningReport(ctypes.Structure):
    _fields_ = [("ncand", ctypes.c_int32), ("best", ctypes.c_int32), ("cand", Tuning * 32)]


class MlpConfig(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("reserved", ctypes.c_int32)]


MLP_NUM_PARAMS = 4929


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("pairs", ctypes.c_int64), ("out_of_history", ctypes.c_int64),
                ("shortcut", ctypes.c_int64), ("bisection", ctypes.c_int64), ("node_tests", ctypes.c_int64),
                ("guard_fallbacks", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("pair_ms", ctypes.c_double),
                ("step_ms", ctypes.c_double), ("timed_steps", ctypes.c_int64), ("dt_last", ctypes.c_double),
                ("eta_min", ctypes.c_double), ("v_max", ctypes.c_double)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_flops", ctypes.c_double), ("fp64_flops", ctypes.c_double), ("mufu_ops", ctypes.c_double),
                ("sms", ctypes.c_int32), ("launches", ctypes.c_int32)]


class AdaptiveDt(ctypes.Structure):
    _fields_ = [("enable", ctypes.c_int32), ("reserved", ctypes.c_int32), ("c_dt", ctypes.c_double),
                ("eta_allow", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double)]


class EnergyMonitor(ctypes.Structure):
    _fields_ = [("enable", ctypes.c_int32), ("hold", ctypes.c_int32), ("eps_E", ctypes.c_double)]


class EnergyState(ctypes.Structure):
    _fields_ = [("ebar", ctypes.c_double), ("rate", ctypes.c_double), ("t_sw", ctypes.c_double),
                ("n_sw", ctypes.c_int64), ("armed", ctypes.c_int32), ("switched", ctypes.c_int32)]


class TwoStageConfig(ctypes.Structure):
    _fields_ = [("eps_E", ctypes.c_double), ("hold", ctypes.c_int32), ("do_handoff", ctypes.c_int32),
                ("max_stage1_steps", ctypes.c_int64), ("check_every", ctypes.c_int64), ("t_after", ctypes.c_double),
                ("bext1", Bext),
                ("center", ctypes.c_double * 3), ("dt2", ctypes.c_double), ("steps2", ctypes.c_int64),
                ("bext2", Bext)]


class TwoStageReport(ctypes.Structure):
    _fields_ = [("n_th", ctypes.c_int64), ("t_th", ctypes.c_double), ("n_sw", ctypes.c_int64), ("t_sw", ctypes.c_double),
                ("stage1_steps_first_run", ctypes.c_int64), ("switched", ctypes.c_int32), ("pad_", ctypes.c_int32)]


EV = 1.602176634e-19  # J per eV (the paper quotes eps_E in keV/s)

_vp = ctypes.c_void_p
_H = ctypes.c_void_p

# name -> (restype, argtypes); every symbol declared in include/emppp.h
SIGNATURES = {
    "emppp_default_options": (None, [ctypes.POINTER(Options)]),
    "emppp_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(Options), _vp,
                                    ctypes.POINTER(_H)]),
    "emppp_create_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                          ctypes.c_double, ctypes.POINTER(Options), _vp, ctypes.POINTER(_H)]),
    "emppp_destroy": (None, [_H]),
    "emppp_handoff": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double)]),
    "emppp_transport": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(Bext)]),
    "emppp_set_particles": (ctypes.c_int, [_H, _vp, _vp, _vp, ctypes.c_int32]),
    "emppp_set_history": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp,
                                         ctypes.c_int32]),
    "emppp_get_history": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), _vp, _vp,
                                         _vp, _vp, ctypes.c_int32]),
    "emppp_step": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.POINTER(Bext)]),
    "emppp_get_state": (ctypes.c_int, [_H, _vp, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.c_int32]),
    "emppp_get_fields": (ctypes.c_int, [_H, _vp, _vp, ctypes.c_int32]),
    "emppp_get_stats": (ctypes.c_int, [_H, ctypes.POINTER(Stats)]),
    "emppp_reset_stats": (ctypes.c_int, [_H]),
    "emppp_set_options": (ctypes.c_int, [_H, ctypes.POINTER(Options)]),
    "emppp_autotune": (ctypes.c_int, [_H, ctypes.POINTER(TuningReport)]),
    "emppp_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(Tuning)]),
    "emppp_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_int32]),
    "emppp_bracket_dump": (ctypes.c_int, [_H, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "emppp_set_stream": (ctypes.c_int, [_H, _vp]),
    "emppp_synchronize": (ctypes.c_int, [_H]),
    "emppp_fields_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "emppp_sample_delays": (ctypes.c_int, [_H, _vp, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_int32]),
    "emppp_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int32, _vp]),
    "emppp_mlp_gradient": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "emppp_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(MlpConfig), _vp, _vp]),
    "emppp_set_proposal": (ctypes.c_int, [_H, _vp, ctypes.c_int32]),
    "emppp_set_adaptive_dt": (ctypes.c_int, [_H, ctypes.POINTER(AdaptiveDt)]),
    "emppp_set_energy_monitor": (ctypes.c_int, [_H, ctypes.POINTER(EnergyMonitor)]),
    "emppp_get_energy": (ctypes.c_int, [_H, ctypes.POINTER(EnergyState)]),
    "emppp_two_stage": (ctypes.c_int, [_H, _vp, _vp, _vp, ctypes.c_int32, ctypes.POINTER(TwoStageConfig),
                                       ctypes.POINTER(TwoStageReport)]),
    "emppp_measure_peaks": (ctypes.c_int, [ctypes.POINTER(Peaks), _vp]),
    "emppp_reciprocal_probe": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    "emppp_last_error": (ctypes.c_char_p, []),
    "emppp_version": (ctypes.c_char_p, []),
}


def library_path() -> str:
    """The library load() uses: the debug build when the environment sets EMPPP_DEBUG_LIB=1."""
    return _build.DEBUG_LIB if os.environ.get("EMPPP_DEBUG_LIB") == "1" else _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (raises if it is not built, unless build_if_missing)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("EMPPP_DEBUG_LIB") == "1"  # the build with the kernels' index range checks
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"EM-PP CUDA library not built ({path}); run __graft_entry__.build()")
        _build.build_library(debug=debug)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != OK:
        raise EmpppError(st, load().emppp_last_error().decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, n_expected, name):
    """(pointer, is_device) of a float64 host array or CUDA tensor with n_expected elements."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch

        if a.dtype != torch.float64 or not a.is_contiguous() or not a.is_cuda:
            raise ValueError(f"{name}: need a contiguous float64 CUDA tensor")
        if a.numel() != n_expected:
            raise ValueError(f"{name}: expected {n_expected} elements, got {a.numel()}")
        return a.data_ptr(), 1
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError(f"{name}: need a C-contiguous float64 numpy array")
    if a.size != n_expected:
        raise ValueError(f"{name}: expected {n_expected} elements, got {a.size}")
    return a.ctypes.data, 0


def _same_kind(*pairs):
    kinds = {k for _, k in pairs if k is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else 0


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def bext_none() -> Bext:
    return Bext(kind=0)


def bext_uniform(b) -> Bext:
    e = Bext(kind=1)
    for c in range(3):
        e.b[c] = float(b[c])
    return e


def bext_dipole(m0: float, center=(0.0, 0.0, 0.0)) -> Bext:
    e = Bext(kind=2, m0=float(m0))
    for c in range(3):
        e.center[c] = float(center[c])
    return e


def make_options(precision="fp64", proposal="bisect", pair_fields=True, source_split=0, timing=False,
                 graphs=True, reconstruction="linear", field_point="present") -> Options:
    o = Options()
    load().emppp_default_options(ctypes.byref(o))
    o.reconstruction = RECONSTRUCTION[reconstruction] if isinstance(reconstruction, str) else int(reconstruction)
    o.field_point = FIELD_POINT[field_point] if isinstance(field_point, str) else int(field_point)
    o.graphs = 1 if graphs else 0
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.proposal = PROPOSAL[proposal] if isinstance(proposal, str) else int(proposal)
    o.pair_fields = 1 if pair_fields else 0
    o.source_split = int(source_split)
    o.timing = 1 if timing else 0
    return o


class Solver:
    """An EM-PP system on one GPU: n particles (or, with `bunches`, several independent bunches whose
    particles are concatenated in every per-particle array), history depth `depth` and step dt."""

    def __init__(self, n: int, depth: int, dt: float, precision="fp64", proposal="bisect", pair_fields=True,
                 source_split=0, stream=None, timing=False, graphs=True, bunches=None, reconstruction="linear",
                 field_point="present"):
        self.lib = load()
        self.depth = int(depth)
        self.dt = float(dt)
        self._h = _H()
        self._opt = make_options(precision, proposal, pair_fields, source_split, timing, graphs, reconstruction,
                                 field_point)
        if bunches is None:
            self.n = int(n)
            self.bunches = [self.n]
            _check(self.lib.emppp_create(self.n, self.depth, self.dt, ctypes.byref(self._opt),
                                         _stream_handle(stream), ctypes.byref(self._h)))
        else:
            self.bunches = [int(b) for b in bunches]
            self.n = sum(self.bunches)
            arr = (ctypes.c_int64 * len(self.bunches))(*self.bunches)
            _check(self.lib.emppp_create_batch(len(self.bunches), arr, self.depth, self.dt, ctypes.byref(self._opt),
                                               _stream_handle(stream), ctypes.byref(self._h)))

    def close(self):
        if self._h:
            self.lib.emppp_destroy(self._h)
            self._h = _H()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_options(self, precision=None, proposal=None, pair_fields=None, source_split=None, timing=None,
                    graphs=None, reconstruction=None, field_point=None):
        o = self._opt
        if reconstruction is not None:
            o.reconstruction = RECONSTRUCTION[reconstruction] if isinstance(reconstruction, str) else int(reconstruction)
        if field_point is not None:
            o.field_point = FIELD_POINT[field_point] if isinstance(field_point, str) else int(field_point)
        if graphs is not None:
            o.graphs = 1 if graphs else 0
        if timing is not None:
            o.timing = 1 if timing else 0
        if precision is not None:
            o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        if proposal is not None:
            o.proposal = PROPOSAL[proposal] if isinstance(proposal, str) else int(proposal)
        if pair_fields is not None:
            o.pair_fields = 1 if pair_fields else 0
        if source_split is not None:
            o.source_split = int(source_split)
        _check(self.lib.emppp_set_options(self._h, ctypes.byref(o)))

    def set_stream(self, stream):
        _check(self.lib.emppp_set_stream(self._h, _stream_handle(stream)))

    def set_particles(self, x, u, w=None):
        px, kx = _ptr(x, 3 * self.n, "x")
        pu, ku = _ptr(u, 3 * self.n, "u")
        pw, kw = _ptr(w, self.n, "w")
        dev = _same_kind((px, kx), (pu, ku), (pw, kw))
        _check(self.lib.emppp_set_particles(self._h, px, pu, pw, dev))

    def set_history(self, n, T, W, V, u, w=None):
        nslots = min(int(n) + 1, self.depth)
        pT, kT = _ptr(T, nslots, "T")
        pW, kW = _ptr(W, nslots * 3 * self.n, "W")
        pV, kV = _ptr(V, nslots * 3 * self.n, "V")
        pu, ku = _ptr(u, 3 * self.n, "u")
        pw, kw = _ptr(w, self.n, "w")
        dev = _same_kind((pT, kT), (pW, kW), (pV, kV), (pu, ku), (pw, kw))
        _check(self.lib.emppp_set_history(self._h, int(n), nslots, pT, pW, pV, pu, pw, dev))

    def get_history(self):
        """(n, T, W, V, u) as numpy arrays (the most recent min(n+1, depth) slots)."""
        T = np.zeros(self.depth)
        W = np.zeros((self.depth, self.n, 3))
        V = np.zeros((self.depth, self.n, 3))
        u = np.zeros((self.n, 3))
        n_now = ctypes.c_int64()
        ns = ctypes.c_int32()
        _check(self.lib.emppp_get_history(self._h, ctypes.byref(n_now), ctypes.byref(ns), T.ctypes.data,
                                          W.ctypes.data, V.ctypes.data, u.ctypes.data, 0))
        k = ns.value
        return n_now.value, T[:k].copy(), W[:k].copy(), V[:k].copy(), u

    def step(self, nsteps=1, bext=None):
        _check(self.lib.emppp_step(self._h, int(nsteps), None if bext is None else ctypes.byref(bext)))

    def handoff(self, center):
        """Translate every bunch so its weighted centroid sits at `center`; history restarts."""
        c = (ctypes.c_double * 3)(*[float(v) for v in center])
        _check(self.lib.emppp_handoff(self._h, c))

    def transport(self, nsteps, dt, bext=None):
        """Stage-2 transport: nsteps steps of dt in the background field only (no pair fields)."""
        _check(self.lib.emppp_transport(self._h, int(nsteps), float(dt), None if bext is None else ctypes.byref(bext)))

    def get_state(self, x=None, u=None):
        """Returns (x, u, t, n). Pass preallocated host arrays or CUDA tensors to fill them in place."""
        if x is None and u is None:
            x = np.zeros((self.n, 3))
            u = np.zeros((self.n, 3))
        px, kx = _ptr(x, 3 * self.n, "x")
        pu, ku = _ptr(u, 3 * self.n, "u")
        dev = _same_kind((px, kx), (pu, ku))
        t = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self.lib.emppp_get_state(self._h, px, pu, ctypes.byref(t), ctypes.byref(n), dev))
        return x, u, t.value, n.value

    def get_fields(self, E=None, B=None):
        if E is None and B is None:
            E = np.zeros((self.n, 3))
            B = np.zeros((self.n, 3))
        pE, kE = _ptr(E, 3 * self.n, "E")
        pB, kB = _ptr(B, 3 * self.n, "B")
        dev = _same_kind((pE, kE), (pB, kB))
        _check(self.lib.emppp_get_fields(self._h, pE, pB, dev))
        return E, B

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib.emppp_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_adaptive_dt(self, enable=True, c_dt=0.05, eta_allow=0.0, dt_min=1e-15, dt_max=1e-12):
        """Adaptive time step of Sec. 2.4 (the paper's C = 0.05 and [1e-15, 1e-12] s by default); enable=False
        returns to the fixed dt."""
        cfg = AdaptiveDt(enable=1 if enable else 0, c_dt=float(c_dt), eta_allow=float(eta_allow), dt_min=float(dt_min),
                         dt_max=float(dt_max))
        _check(self.lib.emppp_set_adaptive_dt(self._h, ctypes.byref(cfg)))

    def set_energy_monitor(self, eps_E, hold=1, enable=True):
        """Stage-switch monitor of Sec. 2.7: eps_E in J/s per electron (30 keV/s = 30e3 * EV)."""
        cfg = EnergyMonitor(enable=1 if enable else 0, hold=int(hold), eps_E=float(eps_E))
        _check(self.lib.emppp_set_energy_monitor(self._h, ctypes.byref(cfg)))

    def get_energy(self) -> list:
        """Per-bunch dicts: ebar (J), rate (J/s), n_sw, t_sw, armed, switched."""
        arr = (EnergyState * len(self.bunches))()
        _check(self.lib.emppp_get_energy(self._h, arr))
        return [{k: getattr(e, k) for k, _ in EnergyState._fields_} for e in arr]

    def two_stage(self, x0, u0, eps_E, max_stage1_steps, dt2, steps2, w0=None, hold=1, check_every=50,
                  t_after=0.0, bext1=None, bext2=None, center=None) -> dict:
        """The two-stage procedure of Sec. 2.7 (emppp_two_stage); center=None skips the handoff."""
        cfg = TwoStageConfig(eps_E=float(eps_E), hold=int(hold), do_handoff=0 if center is None else 1,
                             max_stage1_steps=int(max_stage1_steps), check_every=int(check_every),
                             t_after=float(t_after), dt2=float(dt2), steps2=int(steps2))
        cfg.bext1 = bext1 if bext1 is not None else bext_none()
        cfg.bext2 = bext2 if bext2 is not None else bext_none()
        if center is not None:
            for c in range(3):
                cfg.center[c] = float(center[c])
        px, kx = _ptr(x0, 3 * self.n, "x0")
        pu, ku = _ptr(u0, 3 * self.n, "u0")
        pw, kw = _ptr(w0, self.n, "w0")
        dev = _same_kind((px, kx), (pu, ku), (pw, kw))
        rep = TwoStageReport()
        _check(self.lib.emppp_two_stage(self._h, px, pu, pw, dev, ctypes.byref(cfg), ctypes.byref(rep)))
        return {k: getattr(rep, k) for k, _ in TwoStageReport._fields_ if k != "pad_"}

    def reset_stats(self):
        _check(self.lib.emppp_reset_stats(self._h))

    def autotune(self) -> dict:
        """Time the candidate work splits and tile shapes on the present state and keep the fastest."""
        r = TuningReport()
        _check(self.lib.emppp_autotune(self._h, ctypes.byref(r)))
        cands = [{k: getattr(r.cand[q], k) for k, _ in Tuning._fields_} for q in range(r.ncand)]
        return dict(best=cands[r.best], candidates=cands)

    def bracket_dump(self):
        """(brackets [n, n] int32 numpy array, k0): the bracket 4 (k1 - k0) + branch of every ordered pair of
        the present state (emppp_bracket_dump); -1 on the diagonal and between bunches."""
        import torch

        out = torch.empty((self.n, self.n), dtype=torch.int32, device="cuda")
        k0 = ctypes.c_int64()
        _check(self.lib.emppp_bracket_dump(self._h, out.data_ptr(), ctypes.byref(k0)))
        return out.cpu().numpy(), k0.value

    def set_tuning(self, items_per_block=16, target_order=1, targets_per_block=128, sources_per_sum=8,
                   history_window=0):
        t = Tuning(items_per_block=int(items_per_block), target_order=int(target_order), ms=0.0,
                   targets_per_block=int(targets_per_block), sources_per_sum=int(sources_per_sum),
                   history_window=int(history_window))
        _check(self.lib.emppp_set_tuning(self._h, ctypes.byref(t)))

    def set_wait_limit(self, probes):
        """Probes of a warp's bounded wait on its staged history window (emppp_set_wait_limit)."""
        _check(self.lib.emppp_set_wait_limit(self._h, int(probes)))

    def synchronize(self):
        _check(self.lib.emppp_synchronize(self._h))

    def sample_delays(self, pairs):
        """Features [m, 10], exact delays t - t_r [m] and targets z [m] of (target, source) pairs."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        m = pairs.shape[0]
        feat = np.zeros((m, 10), dtype=np.float32)
        delay = np.zeros(m)
        z = np.zeros(m, dtype=np.float32)
        _check(self.lib.emppp_sample_delays(self._h, pairs.ctypes.data, m, feat.ctypes.data, delay.ctypes.data,
                                            z.ctypes.data, 0))
        return feat, delay, z

    def set_proposal(self, params):
        """Network used by the "mlp" proposal (EMPPP_MLP_NUM_PARAMS float32 values)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_NUM_PARAMS:
            raise ValueError(f"expected {MLP_NUM_PARAMS} parameters")
        _check(self.lib.emppp_set_proposal(self._h, p.ctypes.data, 0))


def fields_noalloc(T, W, V, E, B, w=None, stream=None):
    """Self fields at the present (last) slot of a caller-held device history, computed by the
    library without allocating device memory (see emppp_fields_noalloc in include/emppp.h).
    T [nslots], W, V [nslots, n, 3], E, B [n, 3]: float64 CUDA tensors; w [n] optional."""
    import torch

    tensors = [a for a in (T, W, V, w, E, B) if a is not None]
    if not all(_is_torch(a) and a.is_cuda for a in tensors):
        raise ValueError("fields_noalloc takes device (CUDA tensor) arrays only")
    devices = {a.device for a in tensors}
    if len(devices) != 1:
        raise ValueError(f"fields_noalloc: all arrays must be on one device, got {sorted(map(str, devices))}")
    device = devices.pop()
    if isinstance(stream, torch.cuda.Stream) and stream.device != device:
        raise ValueError(f"fields_noalloc: stream of {stream.device}, arrays on {device}")
    nslots = int(T.numel())
    n = int(W.numel()) // (3 * max(nslots, 1))
    ptrs = [_ptr(T, nslots, "T"), _ptr(W, nslots * 3 * n, "W"), _ptr(V, nslots * 3 * n, "V"),
            _ptr(w, n, "w"), _ptr(E, 3 * n, "E"), _ptr(B, 3 * n, "B")]
    pT, pW, pV, pw, pE, pB = (p for p, _ in ptrs)
    with torch.cuda.device(device):
        _check(load().emppp_fields_noalloc(n, nslots, pT, pW, pV, pw, pE, pB, _stream_handle(stream)))


def _dev_f32(a):
    import torch

    if _is_torch(a):
        return a.to(device="cuda", dtype=torch.float32).contiguous()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def mlp_forward(params, features, mode="reference"):
    """z of the proposal network for features [m, 10] (host arrays or CUDA tensors); returns numpy.
    mode "reference": the form training differentiates; "inference": the form the pair kernels use."""
    import torch

    p, X = _dev_f32(params), _dev_f32(features)
    m = X.shape[0]
    z = torch.empty(m, dtype=torch.float32, device="cuda")
    md = {"reference": 0, "inference": 1}[mode]
    _check(load().emppp_mlp_forward(p.data_ptr(), X.data_ptr(), m, z.data_ptr(), md,
                                    torch.cuda.current_stream().cuda_stream))
    return z.cpu().numpy()


def mlp_gradient(params, features, targets):
    """(mean squared error, gradient [4929]) of one batch."""
    import torch

    p, X, T = _dev_f32(params), _dev_f32(features), _dev_f32(targets)
    g = torch.empty(MLP_NUM_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctypes.c_double()
    _check(load().emppp_mlp_gradient(p.data_ptr(), X.data_ptr(), T.data_ptr(), X.shape[0], g.data_ptr(),
                                     ctypes.byref(loss), torch.cuda.current_stream().cuda_stream))
    return loss.value, g.cpu().numpy()


def mlp_train(params, features, targets, epochs=4, batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              lr_final=0.0):
    """Adam training on the GPU (cosine step-size decay to lr_final when 0 < lr_final < lr); returns
    (trained params as numpy float32, mean loss per epoch)."""
    import torch

    p, X, T = _dev_f32(params).clone(), _dev_f32(features), _dev_f32(targets)
    cfg = MlpConfig(epochs=int(epochs), batch=int(batch), lr=float(lr), beta1=float(beta1), beta2=float(beta2),
                    eps=float(eps), lr_final=float(lr_final))
    losses = np.zeros(max(int(epochs), 1), dtype=np.float32)
    _check(load().emppp_mlp_train(p.data_ptr(), X.data_ptr(), T.data_ptr(), X.shape[0], ctypes.byref(cfg),
                                  losses.ctypes.data, torch.cuda.current_stream().cuda_stream))
    return p.cpu().numpy(), losses[:int(epochs)]


def measure_peaks(stream=None) -> dict:
    """Measured FP32 / FP64 FMA and reciprocal-square-root throughput of the current device
    (emppp_measure_peaks): flop/s, flop/s, operations/s."""
    p = Peaks()
    _check(load().emppp_measure_peaks(ctypes.byref(p), _stream_handle(stream)))
    return {k: getattr(p, k) for k, _ in Peaks._fields_}


def reciprocal_probe(x):
    """1 / x by the FP64 pair kernel's reciprocal, for a float64 CUDA tensor x; returns a CUDA tensor."""
    import torch

    if not (_is_torch(x) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("x: need a contiguous float64 CUDA tensor")
    y = torch.empty_like(x)
    with torch.cuda.device(x.device):
        _check(load().emppp_reciprocal_probe(x.data_ptr(), y.data_ptr(), x.numel(),
                                             torch.cuda.current_stream().cuda_stream))
    return y


def version() -> str:
    return load().emppp_version().decode()
