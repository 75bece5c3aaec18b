"""Plain FP64 CPU oracle for the WENO5-LF / SSP-RK3 shallow-water step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the CUDA product path never
imports it.  The arithmetic lives in ``swe_oracle.c`` (plain C, OpenMP over
independent grid lines only); this module compiles it with gcc and marshals
arguments through ctypes.

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms and invariants the paper fixes (WENO5 polynomial exactness and the
smoothness-indicator definition, fifth-order convergence to the PDE of
Eqs. (1)-(3), lake at rest, mass conservation, mirror and transpose symmetry,
the Stoker dam break of Section 2.1, the planar bowl of Section 2.2, the
Manning normal flow of Section 2.3 and the planar-beach runup law).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_swe.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE = 0, 1, 2, 4


class Params(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_double), ("manning_n", ctypes.c_double), ("h_dry", ctypes.c_double),
        ("h_wet", ctypes.c_double), ("weno_eps", ctypes.c_double), ("fixed_dt", ctypes.c_double),
        ("cfl", ctypes.c_double), ("t_end", ctypes.c_double), ("b_jump_x", ctypes.c_double),
        ("b_jump_y", ctypes.c_double), ("inflow_amp", ctypes.c_double),
        ("inflow_period", ctypes.c_double), ("inflow_depth", ctypes.c_double),
        ("z_ref", ctypes.c_double), ("h_film", ctypes.c_double), ("alpha_margin", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("shore", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


class State(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("last_dt", ctypes.c_double), ("alpha_x", ctypes.c_double),
        ("alpha_y", ctypes.c_double), ("mass", ctypes.c_double), ("clamp_mass", ctypes.c_double),
        ("boundary_mass", ctypes.c_double), ("runup_now", ctypes.c_double),
        ("runup_max", ctypes.c_double), ("steps", ctypes.c_int64), ("status", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile swe_oracle.c into liboracle_swe.so (gcc -O2, OpenMP, no fast-math)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.or_steps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(Params), dp, dp, dp, dp, ctypes.c_int64,
                                 ctypes.POINTER(State)]
        lib.or_steps.restype = ctypes.c_int
        lib.or_diagnose.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(Params), dp, dp, dp, dp, ctypes.POINTER(State)]
        lib.or_diagnose.restype = ctypes.c_int
        lib.or_operator.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(Params), dp, dp, dp, dp, ctypes.c_double,
                                    ctypes.c_double, dp, dp, dp, dp, dp]
        lib.or_operator.restype = ctypes.c_int
        lib.or_operator_split.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(Params), dp, dp, dp, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        lib.or_operator_split.restype = ctypes.c_int
        lib.or_post_stage.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params), dp, dp, dp, dp]
        lib.or_post_stage.restype = ctypes.c_int
        lib.or_weno5.argtypes = [dp, ctypes.c_double, dp]
        lib.or_weno5.restype = ctypes.c_double
        lib.or_inflow_eta.argtypes = [ctypes.POINTER(Params), ctypes.c_double]
        lib.or_inflow_eta.restype = ctypes.c_double
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = None
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params_of(sc) -> Params:
    p = Params()
    p.g, p.manning_n, p.h_dry, p.h_wet = sc.g, sc.manning_n, sc.h_dry, sc.h_wet
    p.weno_eps, p.fixed_dt, p.cfl, p.t_end = sc.weno_eps, sc.fixed_dt, sc.cfl, sc.t_end
    p.b_jump_x, p.b_jump_y = sc.b_jump_x, sc.b_jump_y
    p.inflow_amp, p.inflow_period, p.inflow_depth = sc.inflow_amp, sc.inflow_period, sc.inflow_depth
    p.z_ref = sc.z_ref
    p.h_film = sc.h_film
    p.alpha_margin = sc.alpha_margin
    p.shore = int(sc.shore)
    for k in range(4):
        p.bc[k] = int(sc.bc[k])
    return p


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__("oracle returned status %d" % code)
        self.code = code


class Simulation:
    """A state advanced by the oracle, step by step."""

    def __init__(self, sc):
        self.sc = sc
        self.p = params_of(sc)
        self.b = np.ascontiguousarray(sc.b, dtype=np.float64)
        self.h = np.ascontiguousarray(sc.h, dtype=np.float64).copy()
        self.hu = np.ascontiguousarray(sc.hu, dtype=np.float64).copy()
        self.hv = np.ascontiguousarray(sc.hv, dtype=np.float64).copy()
        self.st = State()
        self.st.t = sc.t0
        self.st.runup_max = -np.inf
        rc = _load().or_diagnose(sc.nx, sc.ny, sc.dx, sc.dy, ctypes.byref(self.p), _dp(self.b), _dp(self.h),
                                 _dp(self.hu), _dp(self.hv), ctypes.byref(self.st))
        if rc:
            raise OracleError(rc)

    def step(self, n: int) -> int:
        """Advance up to n RK3 steps; returns the number taken."""
        before = self.st.steps
        rc = _load().or_steps(self.sc.nx, self.sc.ny, self.sc.dx, self.sc.dy, ctypes.byref(self.p),
                              _dp(self.b), _dp(self.h), _dp(self.hu), _dp(self.hv), int(n),
                              ctypes.byref(self.st))
        if rc:
            raise OracleError(rc)
        return int(self.st.steps - before)

    def run_until(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        old = self.p.t_end
        self.p.t_end = t_end
        try:
            return self.step(max_steps)
        finally:
            self.p.t_end = old

    @property
    def t(self) -> float:
        return float(self.st.t)

    def diag(self) -> Dict[str, float]:
        s = self.st
        return dict(t=s.t, steps=int(s.steps), last_dt=s.last_dt, alpha_x=s.alpha_x, alpha_y=s.alpha_y,
                    mass=s.mass, clamp_mass=s.clamp_mass, boundary_mass=s.boundary_mass,
                    runup_now=s.runup_now, runup_max=s.runup_max)


def operator(sc, t: float = 0.0, dt: float = 0.0, h=None, hu=None, hv=None,
             speeds: Optional[Tuple[float, float]] = None) -> Tuple[np.ndarray, np.ndarray, np.ndarray, Tuple[float, float], float]:
    """One evaluation of the spatial operator L (Eq. (7)) of a state, split
    with the state's own wave speeds, or with `speeds` = (alpha_x, alpha_y)."""
    p = params_of(sc)
    b = np.ascontiguousarray(sc.b, dtype=np.float64)
    h = np.ascontiguousarray(sc.h if h is None else h, dtype=np.float64)
    hu = np.ascontiguousarray(sc.hu if hu is None else hu, dtype=np.float64)
    hv = np.ascontiguousarray(sc.hv if hv is None else hv, dtype=np.float64)
    Lh, Lhu, Lhv = (np.zeros_like(b) for _ in range(3))
    a2 = np.zeros(2)
    ef = np.zeros(1)
    lib = _load()
    if speeds is None:
        rc = lib.or_operator(sc.nx, sc.ny, sc.dx, sc.dy, ctypes.byref(p), _dp(b), _dp(h), _dp(hu), _dp(hv),
                             float(t), float(dt), _dp(Lh), _dp(Lhu), _dp(Lhv), _dp(a2), _dp(ef))
    else:
        a2[:] = speeds
        rc = lib.or_operator_split(sc.nx, sc.ny, sc.dx, sc.dy, ctypes.byref(p), _dp(b), _dp(h), _dp(hu),
                                   _dp(hv), float(t), float(dt), float(a2[0]), float(a2[1]), _dp(Lh),
                                   _dp(Lhu), _dp(Lhv), _dp(ef))
    if rc:
        raise OracleError(rc)
    return Lh, Lhu, Lhv, (float(a2[0]), float(a2[1])), float(ef[0])


def post_stage(sc, h, hu, hv) -> Tuple[np.ndarray, np.ndarray, np.ndarray, float]:
    """The post-stage rule of every RK stage applied once to a state (R5 and
    the film desingularisation): returns the new (h, hu, hv) and the depth
    added by the h < 0 clamp, summed over cells."""
    p = params_of(sc)
    h, hu, hv = (np.array(x, dtype=np.float64, order="C") for x in (h, hu, hv))
    ny, nx = h.shape
    added = np.zeros(1)
    rc = _load().or_post_stage(nx, ny, ctypes.byref(p), _dp(h), _dp(hu), _dp(hv), _dp(added))
    if rc:
        raise OracleError(rc)
    return h, hu, hv, float(added[0])


def weno5(v, eps: float = 1e-6) -> Tuple[float, np.ndarray]:
    """WENO5-JS value at the right face of v[2] and its nonlinear weights."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (5,)
    w = np.zeros(3)
    r = _load().or_weno5(_dp(v), float(eps), _dp(w))
    return float(r), w


def inflow_eta(sc, t: float) -> float:
    p = params_of(sc)
    return float(_load().or_inflow_eta(ctypes.byref(p), float(t)))


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_threads(n: int) -> None:
    """Threads of the grid-line loops (timing at 1 thread and at all cores);
    does not change the arithmetic."""
    _load().or_set_threads(int(n))


def run(sc, steps: Optional[int] = None) -> Simulation:
    sim = Simulation(sc)
    sim.step(sc.steps if steps is None else steps)
    return sim
