"""EM-PP oracle -- test infrastructure only.

A plain, slow FP64 CPU statement of one EM-PP step of arXiv 2605.05543 (Sec. 2.1 Lienard-Wiechert
fields and superposition, Sec. 2.2 retarded-time bracketing and linear reconstruction, Sec. 2.3
Higuera-Cary push, Sec. 2.6 dipole background field), in ``emppp_oracle.c``, plus the MLP
reference of ``mlp.py``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It shares no code with the CUDA library and never imports it.

History layout used throughout: ``T[k]`` (s), ``W[k, j, :]`` (m) and ``V[k, j, :]`` (m/s) for slots
``k = 0..n``; the depth ``D`` sets the earliest usable slot ``k0 = max(0, n - D + 1)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emppp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "liboracle.so")

_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)

BRANCH_NAMES = ("out_of_history", "shortcut", "bisection")


def compile_lib(src: str = _SRC, out: str = _LIBPATH, openmp: bool = True, extra=()) -> str:
    """Compile the oracle C source into a shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    if openmp:
        cmd.append("-fopenmp")
    cmd += list(extra) + [src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build() -> str:
    """Build the oracle library in-tree if it is missing or older than its source."""
    if not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        compile_lib()
    return _LIBPATH


def _bind(lib):
    lib.orc_constants.argtypes = [_d]
    lib.orc_num_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_lw_fields.argtypes = [_d, _d, _d, ctypes.c_double, _d, _d]
    lib.orc_lw_fields.restype = ctypes.c_int
    lib.orc_background_b.argtypes = [ctypes.c_int, _d, _d, _d]
    lib.orc_hc_kick.argtypes = [_d, _d, _d, ctypes.c_double, _d]
    lib.orc_node_test.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_int64, _d, ctypes.c_double, ctypes.c_int64]
    lib.orc_node_test.restype = ctypes.c_int
    lib.orc_retarded.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 _d, _d, _d, _i64]
    lib.orc_retarded.restype = ctypes.c_int
    lib.orc_retarded_ex.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                    _d, ctypes.c_int, _d, _d, _i64]
    lib.orc_retarded_ex.restype = ctypes.c_int
    lib.orc_bracket_table.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int32)]
    lib.orc_bracket_table.restype = ctypes.c_int
    lib.orc_self_fields.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, _d, _i64,
                                    ctypes.c_int64, _d, _d, _d, _i64]
    lib.orc_self_fields.restype = ctypes.c_int
    lib.orc_self_fields_ex.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, _d, _i64,
                                       ctypes.c_int64, ctypes.c_int, _d, _d, _d, _i64]
    lib.orc_self_fields_ex.restype = ctypes.c_int
    lib.orc_push.argtypes = [ctypes.c_int64, ctypes.c_double, _d, _d, _d, _d, ctypes.c_int, _d, _d, _d]
    lib.orc_push.restype = ctypes.c_int
    lib.orc_step.argtypes = [ctypes.c_int64, _d, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                             _d, ctypes.c_int, _d, ctypes.c_int, _d, _d, _i64]
    lib.orc_step.restype = ctypes.c_int
    lib.orc_step_ex.argtypes = [ctypes.c_int64, _d, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                _d, ctypes.c_int, _d, ctypes.c_int, ctypes.c_int, _d, _d, _i64]
    lib.orc_step_ex.restype = ctypes.c_int
    lib.orc_interaction_scale.argtypes = [ctypes.c_int64, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                          _d]
    lib.orc_interaction_scale.restype = ctypes.c_int
    lib.orc_adaptive_dt.argtypes = [ctypes.c_double] * 5
    lib.orc_adaptive_dt.restype = ctypes.c_double
    lib.orc_step_adaptive.argtypes = [ctypes.c_int64, _d, _d, _d, _d, ctypes.c_int64, ctypes.c_int64, _d, _d,
                                      ctypes.c_int, _d, _d, _d, _i64, _d]
    lib.orc_step_adaptive.restype = ctypes.c_int
    lib.orc_mean_kinetic_energy.argtypes = [ctypes.c_int64, _d, _d]
    lib.orc_mean_kinetic_energy.restype = ctypes.c_double
    lib.orc_energy_switch.argtypes = [ctypes.c_int64, _d, _d, ctypes.c_double, ctypes.c_int64, _d]
    lib.orc_energy_switch.restype = ctypes.c_int64
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library. A custom path loads a separate copy."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _p(a):
    return a.ctypes.data_as(_d)


def _pi(a):
    return a.ctypes.data_as(_i64)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def constants(lib=None) -> dict:
    """CODATA 2018 constants used by the oracle."""
    lib = lib or load()
    out = np.zeros(5)
    lib.orc_constants(_p(out))
    return dict(c=out[0], e=out[1], m_e=out[2], eps0=out[3], mu0=out[4])


def set_threads(n: int, lib=None):
    (lib or load()).orc_set_threads(int(n))


def num_threads(lib=None) -> int:
    return int((lib or load()).orc_num_threads())


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"oracle {what} failed with status {st}")


def lw_fields(eta, v, a, q, lib=None):
    """eq:LW_E / eq:LW_B for one source: returns (E, B)."""
    lib = lib or load()
    eta, v, a = _f64(eta, 3), _f64(v, 3), _f64(a, 3)
    E, B = np.zeros(3), np.zeros(3)
    _check(lib.orc_lw_fields(_p(eta), _p(v), _p(a), float(q), _p(E), _p(B)), "lw_fields")
    return E, B


def bext_params(kind: int = 0, b=(0.0, 0.0, 0.0), m0: float = 0.0, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    return np.array([b[0], b[1], b[2], m0, center[0], center[1], center[2]], dtype=np.float64)


def background_b(kind, par, x, lib=None):
    lib = lib or load()
    par, x = _f64(par, 7), _f64(x, 3)
    B = np.zeros(3)
    lib.orc_background_b(int(kind), _p(par), _p(x), _p(B))
    return B


def hc_kick(u, E, B, h, lib=None):
    """One Higuera-Cary proper-velocity update with h = q dt / (2 m)."""
    lib = lib or load()
    u, E, B = _f64(u, 3), _f64(E, 3), _f64(B, 3)
    out = np.zeros(3)
    lib.orc_hc_kick(_p(u), _p(E), _p(B), float(h), _p(out))
    return out


def node_test(T, W, j, r, t, k, lib=None) -> bool:
    lib = lib or load()
    T, W, r = _f64(T), _f64(W), _f64(r, 3)
    return bool(lib.orc_node_test(W.shape[1], _p(T), _p(W), int(j), _p(r), float(t), int(k)))


# step variants, kept as accuracy comparisons: the midpoint reconstruction of eq:mid and the self fields
# at the half-step point (x^{n+1/2}, t_n + dt/2)
MIDPOINT = 1
HALF_STEP = 2


def retarded(T, W, V, n, D, j, r, lib=None, variant=0):
    """Retarded state of source j seen from (r, T[n]): dict(w, v, a, tr, branch, k1, ntest).
    variant = MIDPOINT reconstructs bracketed pairs by eq:mid."""
    lib = lib or load()
    T, W, V, r = _f64(T), _f64(W), _f64(V), _f64(r, 3)
    out = np.zeros(9)
    tr = np.zeros(1)
    info = np.zeros(3, dtype=np.int64)
    st = lib.orc_retarded_ex(W.shape[1], _p(T), _p(W), _p(V), int(n), int(D), int(j), _p(r), int(variant),
                             _p(out), _p(tr), _pi(info))
    _check(st, "retarded")
    return dict(w=out[0:3].copy(), v=out[3:6].copy(), a=out[6:9].copy(), tr=float(tr[0]),
                branch=int(info[0]), k1=int(info[1]), ntest=int(info[2]))


def bracket_table(T, W, n, D, lib=None):
    """Brackets of all ordered pairs at step n (Sec. 2.2 search): int32 [N, N] with 4 (k1 - k0) + branch
    for j != i (k0 = max(0, n - D + 1)) and -1 on the diagonal."""
    lib = lib or load()
    T, W = _f64(T), _f64(W)
    N = W.shape[1]
    out = np.zeros((N, N), dtype=np.int32)
    _check(lib.orc_bracket_table(N, _p(T), _p(W), int(n), int(D), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "bracket_table")
    return out


def self_fields(T, W, V, n, D, weights=None, targets=None, lib=None, mags=False, variant=0):
    """Self fields on targets (all if None) at step n. Returns (E, B, stats), or (E, B, stats, M) with
    mags=True where M[:, 0] = sum_j |E_ij| and M[:, 1] = sum_j |B_ij| per target. variant = MIDPOINT
    reconstructs bracketed pairs by eq:mid.

    stats = dict(out_of_history, shortcut, bisection, node_tests) over all evaluated pairs.
    """
    lib = lib or load()
    T, W, V = _f64(T), _f64(W), _f64(V)
    N = W.shape[1]
    wts = None if weights is None else _f64(weights)
    if targets is None:
        nt = N
        tg = None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tg.shape[0]
    E = np.zeros((nt, 3))
    B = np.zeros((nt, 3))
    stats = np.zeros(4, dtype=np.int64)
    M = np.zeros((nt, 2))
    st = lib.orc_self_fields_ex(N, _p(T), _p(W), _p(V), int(n), int(D), None if wts is None else _p(wts),
                                None if tg is None else _pi(tg), nt, int(variant), _p(E), _p(B), _p(M), _pi(stats))
    _check(st, "self_fields")
    sd = dict(zip(("out_of_history", "shortcut", "bisection", "node_tests"), stats.tolist()))
    return (E, B, sd, M) if mags else (E, B, sd)


def interaction_scale(T, W, V, n, D, eta_allow=0.0, lib=None):
    """(eta_min, v_max) of the adaptive time step (Sec. 2.4) at step n."""
    lib = lib or load()
    T, W, V = _f64(T), _f64(W), _f64(V)
    out = np.zeros(2)
    _check(lib.orc_interaction_scale(W.shape[1], _p(T), _p(W), _p(V), int(n), int(D), float(eta_allow), _p(out)),
           "interaction_scale")
    return float(out[0]), float(out[1])


def adaptive_dt(eta_min, v_max, c_dt=0.05, dt_min=1e-15, dt_max=1e-12, lib=None):
    """dt = c_dt eta_min / v_max clamped to [dt_min, dt_max] (Sec. 2.4)."""
    lib = lib or load()
    return float(lib.orc_adaptive_dt(float(eta_min), float(v_max), float(c_dt), float(dt_min), float(dt_max)))


ADAPTIVE_PAPER = dict(c_dt=0.05, eta_allow=0.0, dt_min=1e-15, dt_max=1e-12)


def mean_kinetic_energy(u, weights=None, lib=None):
    """Weighted mean kinetic energy per electron (J) of Sec. 2.7."""
    lib = lib or load()
    u = _f64(u)
    w = None if weights is None else _f64(weights)
    return float(lib.orc_mean_kinetic_energy(u.shape[0], _p(u), None if w is None else _p(w)))


def energy_switch(T, E, eps, hold=1, lib=None):
    """(n_sw, rates) of the switching criterion |dE/dt| < eps of Sec. 2.7 on a record E(T); n_sw = -1
    when the criterion never holds for `hold` consecutive steps."""
    lib = lib or load()
    T, E = _f64(T), _f64(E)
    rate = np.zeros(T.shape[0])
    n = int(lib.orc_energy_switch(T.shape[0], _p(T), _p(E), float(eps), int(hold), _p(rate)))
    return n, rate


def push(x, u, E, B, dt, bkind=0, bpar=None, lib=None):
    """The push of Sec. 2.3 for the given particles with the given self fields (drift dt/2, background
    field at the half-step position, Higuera-Cary kick, drift dt/2). Returns (x_new, u_new, B_total)."""
    lib = lib or load()
    x, u, E, B = (_f64(a).reshape(-1, 3).copy() for a in (x, u, E, B))
    bpar = bext_params() if bpar is None else _f64(bpar, 7)
    v = np.zeros_like(x)
    Bt = np.zeros_like(x)
    _check(lib.orc_push(x.shape[0], float(dt), _p(x), _p(u), _p(E), _p(B), int(bkind), _p(bpar), _p(v), _p(Bt)),
           "push")
    return x, u, Bt


def velocity(u):
    """v = u / gamma with gamma = sqrt(1 + u.u / c^2), the way the oracle forms it."""
    c = constants()["c"]
    u = _f64(u)
    uu = u[..., 0] * u[..., 0] + u[..., 1] * u[..., 1] + u[..., 2] * u[..., 2]
    g = np.sqrt(1.0 + uu / (c * c))
    return u / g[..., None]


class Run:
    """A full oracle simulation: history arrays with room for ``nmax`` slots after the start."""

    def __init__(self, x0, u0, D, dt, weights=None, nmax=0, T0=None, W0=None, V0=None, t0=0.0, lib=None):
        self.lib = lib or load()
        u0 = _f64(u0)
        self.N = u0.shape[0]
        self.D = int(D)
        self.dt = float(dt)
        self.weights = None if weights is None else _f64(weights)
        if W0 is None:
            x0 = _f64(x0)
            W0 = x0[None]
            V0 = velocity(u0)[None]
            T0 = np.array([t0])
        nh = W0.shape[0]
        S = nh + int(nmax)
        self.T = np.zeros(S)
        self.W = np.zeros((S, self.N, 3))
        self.V = np.zeros((S, self.N, 3))
        self.T[:nh] = T0
        self.W[:nh] = W0
        self.V[:nh] = V0
        self.n = nh - 1
        self.u = u0.copy()
        self.E = None
        self.B = None
        self.stats = None
        self.adaptive_log = []

    @property
    def x(self):
        return self.W[self.n]

    @property
    def t(self):
        return self.T[self.n]

    def step(self, nsteps=1, bkind=0, bpar=None, self_on=True, adaptive=None, variant=0):
        """nsteps steps; adaptive = dict(c_dt, eta_allow, dt_min, dt_max) chooses each step's dt by the
        rule of Sec. 2.4 (self fields on) and appends (dt, eta_min, v_max) to self.adaptive_log.
        variant (fixed dt only): MIDPOINT and/or HALF_STEP, the comparison variants of the step."""
        if adaptive is not None and variant:
            raise OracleError("the step variants run with a fixed dt")
        bpar = bext_params() if bpar is None else _f64(bpar, 7)
        E = np.zeros((self.N, 3))
        B = np.zeros((self.N, 3))
        stats = np.zeros(4, dtype=np.int64)
        wp = None if self.weights is None else _p(self.weights)
        if adaptive is not None:
            par = np.array([adaptive["c_dt"], adaptive["eta_allow"], adaptive["dt_min"], adaptive["dt_max"]], dtype=float)
            info = np.zeros(3)
        for _ in range(int(nsteps)):
            if self.n + 1 >= self.T.shape[0]:
                raise OracleError("history capacity exhausted")
            if adaptive is None:
                st = self.lib.orc_step_ex(self.N, _p(self.T), _p(self.W), _p(self.V), _p(self.u), self.n, self.D,
                                          self.dt, wp, int(bkind), _p(bpar), 1 if self_on else 0, int(variant), _p(E),
                                          _p(B), _pi(stats))
            else:
                st = self.lib.orc_step_adaptive(self.N, _p(self.T), _p(self.W), _p(self.V), _p(self.u), self.n,
                                                self.D, _p(par), wp, int(bkind), _p(bpar), _p(E), _p(B), _pi(stats),
                                                _p(info))
                self.adaptive_log.append(tuple(info.tolist()))
            _check(st, "step")
            self.n += 1
        self.E, self.B = E, B
        self.stats = dict(zip(("out_of_history", "shortcut", "bisection", "node_tests"), stats.tolist()))
        return self


def self_test_build() -> None:
    """Raise if the oracle library cannot be built and loaded."""
    lib = load()
    constants(lib)
    print(f"oracle loaded from {_LIBPATH} ({num_threads(lib)} threads)", file=sys.stderr)
