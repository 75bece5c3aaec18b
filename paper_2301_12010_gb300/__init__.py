"""GB300 (sm_103a) solver for the 2-D nonlinear shallow-water equations with
WENO5 / global Lax-Friedrichs flux splitting and SSP-RK3 (the method of
arXiv:2301.12010, "Numerical approximation").

This module is a thin ctypes binding over the C ABI of ``libswe.so``
(declared in ``include/swe.h``): it marshals arguments and nothing else.
Every step of the solver runs in the library's CUDA kernels; there is no
CPU fallback.  If the library is missing the import fails loudly; build it
with ``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# SWE_LIB_VARIANT=checked loads the index-checked build (libswe_checked.so)
LIB_PATH = os.path.join(_PKG, "libswe_checked.so" if os.environ.get("SWE_LIB_VARIANT") == "checked"
                        else "libswe.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EBUDGET, EFULL = range(8)
F32, F64 = 0, 1
WALL, INFLOW, PERIODIC = 0, 1, 2


class SweError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _strerror(code)
        super().__init__("%s: %s (status %d)" % (what, msg, code) if what else "%s (status %d)" % (msg, code))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_double), ("manning_n", ctypes.c_double), ("h_dry", ctypes.c_double),
        ("h_wet", ctypes.c_double), ("h_film", ctypes.c_double), ("weno_eps", ctypes.c_double),
        ("fixed_dt", ctypes.c_double), ("z_ref", ctypes.c_double), ("b_jump_x", ctypes.c_double), ("b_jump_y", ctypes.c_double),
        ("inflow_amp", ctypes.c_double), ("inflow_period", ctypes.c_double), ("inflow_depth", ctypes.c_double),
        ("alpha_margin", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("precision", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("fused_step", ctypes.c_int32), ("shore", ctypes.c_int32), ("stream", ctypes.c_void_p),
    ]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class Diag(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("steps", ctypes.c_int64), ("last_dt", ctypes.c_double),
        ("alpha_x", ctypes.c_double), ("alpha_y", ctypes.c_double), ("clamp_mass", ctypes.c_double),
        ("boundary_mass", ctypes.c_double), ("runup_now", ctypes.c_double), ("runup_max", ctypes.c_double),
        ("status", ctypes.c_int32), ("tile", ctypes.c_int32),
    ]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("libswe.so is not built (%s); run __graft_entry__.build() on a machine with nvcc"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    H = ctypes.c_void_p
    sig = {
        "swe_params_default": (None, [ctypes.POINTER(Params)]),
        "swe_create": (ip, [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(Params),
                            ctypes.POINTER(H)]),
        "swe_set_state": (ip, [H, dp, dp, dp]),
        "swe_set_state_device": (ip, [H, vp, vp, vp]),
        "swe_set_state_async": (ip, [H, dp, dp, dp]),
        "swe_step": (ip, [H, ctypes.c_int32, ctypes.c_double]),
        "swe_sync": (ip, [H]),
        "swe_get_state": (ip, [H, dp, dp, dp]),
        "swe_get_state_async": (ip, [H, dp, dp, dp]),
        "swe_wait_state": (ip, [H]),
        "swe_set_horizon": (ip, [H, ctypes.c_double]),
        "swe_set_wait": (ip, [H, ctypes.c_double, ctypes.c_int32]),
        "swe_get_state_device": (ip, [H, vp, vp, vp]),
        "swe_mass": (ip, [H, dp, dp]),
        "swe_runup": (ip, [H, dp, dp]),
        "swe_get_time": (ip, [H, dp, ctypes.POINTER(ctypes.c_int64)]),
        "swe_set_time": (ip, [H, ctypes.c_double]),
        "swe_diagnostics": (ip, [H, ctypes.POINTER(Diag)]),
        "swe_status": (ip, [H]),
        "swe_strerror": (ctypes.c_char_p, [ip]),
        "swe_destroy": (ip, [H]),
        "swe_tile_count": (ip, []),
        "swe_tile_shape": (ip, [ip, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int32)]),
        "swe_time_stages": (ip, [H, ctypes.c_int32, ctypes.c_double, dp, dp]),
        "swe_batch_slot_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid)]),
        "swe_batch_create": (ip, [ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(Params), ctypes.POINTER(H)]),
        "swe_batch_admit": (ip, [H, ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                 ctypes.c_double, ctypes.POINTER(ctypes.c_int32)]),
        "swe_batch_run": (ip, [H, ctypes.c_int32, ctypes.c_double]),
        "swe_batch_poll": (ip, [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "swe_batch_select": (ip, [H, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
        "swe_batch_times": (ip, [H, dp]),
        "swe_batch_set_time": (ip, [H, ctypes.c_int32, ctypes.c_double]),
        "swe_batch_get_state": (ip, [H, ctypes.c_int32, dp, dp, dp]),
        "swe_batch_diagnostics": (ip, [H, ctypes.c_int32, ctypes.POINTER(Diag)]),
        "swe_batch_retire": (ip, [H, ctypes.c_int32, dp, dp, dp, dp, dp]),
        "swe_batch_memory": (ip, [H, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
        "swe_batch_status": (ip, [H]),
        "swe_batch_set_barrier": (ip, [H, ctypes.c_double, ctypes.c_int32]),
        "swe_batch_destroy": (ip, [H]),
        "swe_autotune": (ip, [ctypes.POINTER(Grid), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_int32), dp]),
        "swe_autotune_lookup": (ip, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double]),
        "swe_debug_fail_alloc": (ip, [ctypes.c_int32]),
        "swe_checked_build": (ip, []),
        "swe_strip_bounds": (ip, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32)]),
        "swe_multi_create": (ip, [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, dp, ctypes.POINTER(Params),
                                  ctypes.c_int32, ctypes.POINTER(H)]),
        "swe_multi_set_state": (ip, [H, dp, dp, dp]),
        "swe_multi_set_time": (ip, [H, ctypes.c_double]),
        "swe_multi_step": (ip, [H, ctypes.c_int32, ctypes.c_double]),
        "swe_multi_get_state": (ip, [H, dp, dp, dp]),
        "swe_multi_mass": (ip, [H, dp]),
        "swe_multi_diagnostics": (ip, [H, ctypes.POINTER(Diag)]),
        "swe_multi_destroy": (ip, [H]),
        "swe_check_status": (ip, [H, ctypes.POINTER(ctypes.c_uint64)]),
        "swe_batch_check_status": (ip, [H, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _strerror(code: int) -> str:
    return lib.swe_strerror(int(code)).decode()


def _check(rc: int, what: str = "") -> None:
    if rc != OK:
        raise SweError(rc, what)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def debug_fail_alloc(n: int) -> None:
    """Test hook (swe_debug_fail_alloc): the n-th device allocation of the
    library from now on fails with ENOMEM; 0 disarms."""
    _check(lib.swe_debug_fail_alloc(int(n)), "swe_debug_fail_alloc")


def tile_shapes() -> Sequence[Tuple[int, int, int]]:
    out = []
    for k in range(1, lib.swe_tile_count() + 1):
        tx, ty, nt = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.swe_tile_shape(k, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(nt)))
        out.append((tx.value, ty.value, nt.value))
    return out


def params_for(sc, precision: int = F32, stream: Optional[int] = None, tile: int = 0) -> Params:
    """swe_params from a workload description (any object with the fields)."""
    p = Params()
    lib.swe_params_default(ctypes.byref(p))
    p.g, p.manning_n, p.h_dry, p.h_wet, p.h_film = sc.g, sc.manning_n, sc.h_dry, sc.h_wet, sc.h_film
    p.weno_eps, p.fixed_dt, p.z_ref = sc.weno_eps, sc.fixed_dt, sc.z_ref
    p.b_jump_x, p.b_jump_y = sc.b_jump_x, sc.b_jump_y
    p.inflow_amp, p.inflow_period, p.inflow_depth = sc.inflow_amp, sc.inflow_period, sc.inflow_depth
    for k in range(4):
        p.bc[k] = int(sc.bc[k])
    p.shore = int(getattr(sc, "shore", 0) or 0)  # the shoreline variant
    margin = float(getattr(sc, "alpha_margin", 0.0) or 0.0)
    if margin > 0.0:  # the fused-step variant (one splitting speed per step)
        p.fused_step = 1
        p.alpha_margin = margin
    p.precision = int(precision)
    p.tile = int(tile)
    p.stream = stream
    return p


class Solver:
    """One scenario on the GPU, driven through the C ABI."""

    def __init__(self, sc, precision: int = F32, stream: Optional[int] = None, tile: int = 0,
                 set_state: bool = True):
        self.sc = sc
        self.precision = precision
        self.nx, self.ny = sc.nx, sc.ny
        self._h = ctypes.c_void_p()
        self._async_in, self._async_out = [], []  # host arrays of uploads and read-backs in flight
        b = np.ascontiguousarray(sc.b, dtype=np.float64)
        g = Grid(sc.nx, sc.ny)
        self.params = params_for(sc, precision, stream, tile)
        _check(lib.swe_create(ctypes.byref(g), float(sc.dx), float(sc.dy), _dp(b), ctypes.byref(self.params),
                              ctypes.byref(self._h)), "swe_create")
        if sc.t0:
            _check(lib.swe_set_time(self._h, float(sc.t0)), "swe_set_time")
        if set_state:
            self.set_state(sc.h, sc.hu, sc.hv)

    # -- life cycle
    def close(self) -> None:
        if self._h:
            lib.swe_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- state
    def set_state(self, h, hu, hv) -> None:
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (h, hu, hv)]
        _check(lib.swe_set_state(self._h, *[_dp(x) for x in a]), "swe_set_state")

    def set_state_async(self, h, hu, hv) -> None:
        """Upload a state from page-locked float64 arrays without waiting
        (swe_set_state_async); the arrays must stay unchanged until the next
        synchronising call.  Pageable arrays are uploaded synchronously."""
        for x in (h, hu, hv):
            if x.dtype != np.float64 or not x.flags.c_contiguous or x.shape != (self.ny, self.nx):
                raise ValueError("set_state_async needs contiguous float64 arrays of shape (ny, nx)")
        self._async_in.append((h, hu, hv))  # kept alive until the stream is synchronised
        _check(lib.swe_set_state_async(self._h, *[_dp(x) for x in (h, hu, hv)]), "swe_set_state_async")

    def set_state_device(self, h, hu, hv) -> None:
        """From device tensors (torch) of the solver's precision, contiguous [ny][nx]."""
        _check(lib.swe_set_state_device(self._h, h.data_ptr(), hu.data_ptr(), hv.data_ptr()),
               "swe_set_state_device")

    def get_state(self, out=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        if out is None:
            out = tuple(np.empty((self.ny, self.nx), dtype=np.float64) for _ in range(3))
        _check(lib.swe_get_state(self._h, *[_dp(x) for x in out]), "swe_get_state")
        self._async_in = []  # the stream is synchronised
        return out

    def get_state_async(self, out) -> None:
        """Start the read-back of the state into `out` (three contiguous
        float64 arrays, page-locked for the asynchronous path); the arrays
        hold the state once wait_state() returns."""
        for x in out:
            if x.dtype != np.float64 or not x.flags.c_contiguous or x.shape != (self.ny, self.nx):
                raise ValueError("get_state_async needs contiguous float64 arrays of shape (ny, nx)")
        self._async_out.append(out)  # kept alive until wait_state
        _check(lib.swe_get_state_async(self._h, *[_dp(x) for x in out]), "swe_get_state_async")

    def set_wait(self, timeout_s: float = 1.0, extra_copy_bytes: int = 0) -> None:
        """Bounded waits of the halo-box copies (see swe_set_wait); a positive
        extra_copy_bytes is a test hook that makes the waits run out."""
        _check(lib.swe_set_wait(self._h, float(timeout_s), int(extra_copy_bytes)), "swe_set_wait")

    def wait_state(self) -> None:
        _check(lib.swe_wait_state(self._h), "swe_wait_state")
        self._async_out = []

    def get_state_device(self, h, hu, hv) -> None:
        _check(lib.swe_get_state_device(self._h, h.data_ptr(), hu.data_ptr(), hv.data_ptr()),
               "swe_get_state_device")

    # -- stepping
    def step(self, n: int, cfl: Optional[float] = None) -> None:
        c = self.sc.cfl if cfl is None else cfl
        _check(lib.swe_step(self._h, int(n), float(c)), "swe_step")

    def sync(self) -> None:
        _check(lib.swe_sync(self._h), "swe_sync")
        self._async_in = []

    def status(self) -> int:
        return int(lib.swe_status(self._h))

    def check_word(self) -> int:
        """Checked build: the first out-of-range index recorded (0: none)."""
        w = ctypes.c_uint64()
        _check(lib.swe_check_status(self._h, ctypes.byref(w)), "swe_check_status")
        return int(w.value)

    def set_time(self, t: float) -> None:
        _check(lib.swe_set_time(self._h, float(t)), "swe_set_time")

    def set_horizon(self, t_end: float) -> None:
        """Stop at simulated time t_end (the last step shortened to end on
        it, later steps doing nothing); 0 removes the horizon."""
        _check(lib.swe_set_horizon(self._h, float(t_end)), "swe_set_horizon")

    # -- diagnostics
    def diagnostics(self, check: bool = True) -> Dict[str, float]:
        d = Diag()
        rc = lib.swe_diagnostics(self._h, ctypes.byref(d))
        if check:
            _check(rc, "swe_diagnostics")
        return dict(t=d.t, steps=int(d.steps), last_dt=d.last_dt, alpha_x=d.alpha_x, alpha_y=d.alpha_y,
                    clamp_mass=d.clamp_mass, boundary_mass=d.boundary_mass, runup_now=d.runup_now,
                    runup_max=d.runup_max, status=int(d.status), tile=int(d.tile))

    def mass(self) -> Tuple[float, float]:
        m, c = ctypes.c_double(), ctypes.c_double()
        _check(lib.swe_mass(self._h, ctypes.byref(m), ctypes.byref(c)), "swe_mass")
        return m.value, c.value

    def runup(self) -> Tuple[float, float]:
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib.swe_runup(self._h, ctypes.byref(a), ctypes.byref(b)), "swe_runup")
        return a.value, b.value

    def time(self) -> Tuple[float, int]:
        t, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib.swe_get_time(self._h, ctypes.byref(t), ctypes.byref(n)), "swe_get_time")
        return t.value, int(n.value)

    def time_stages(self, n: int, cfl: Optional[float] = None) -> Tuple[float, Tuple[float, float, float]]:
        c = self.sc.cfl if cfl is None else cfl
        tot = ctypes.c_double()
        st = (ctypes.c_double * 3)()
        _check(lib.swe_time_stages(self._h, int(n), float(c), ctypes.byref(tot), st), "swe_time_stages")
        return tot.value, (st[0], st[1], st[2])


def _diag_dict(d: Diag) -> Dict[str, float]:
    return dict(t=d.t, steps=int(d.steps), last_dt=d.last_dt, alpha_x=d.alpha_x, alpha_y=d.alpha_y,
                clamp_mass=d.clamp_mass, boundary_mass=d.boundary_mass, runup_now=d.runup_now,
                runup_max=d.runup_max, status=int(d.status), tile=int(d.tile))


def autotune(shapes, precision: int = F32, batch: bool = False, steps: int = 10):
    """Time every compiled tile shape (C++ timing loop) on synthetic scenarios
    of the given (nx, ny) grid sizes; the winner goes to the autotune cache and
    is used by Solver / Batch created with tile=0.  Returns (best, ms_per_step)."""
    grids = (Grid * len(shapes))(*[Grid(int(nx), int(ny)) for nx, ny in shapes])
    best = ctypes.c_int32()
    ms = (ctypes.c_double * lib.swe_tile_count())()
    _check(lib.swe_autotune(grids, len(shapes), int(precision), 1 if batch else 0, int(steps), ctypes.byref(best), ms),
           "swe_autotune")
    return best.value, list(ms)


def strip_bounds(ny: int, nparts: int):
    """[(first row, rows)] of the row partition swe_multi uses (host only)."""
    out = []
    for k in range(int(nparts)):
        r0, n = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.swe_strip_bounds(int(ny), int(nparts), k, ctypes.byref(r0), ctypes.byref(n)), "swe_strip_bounds")
        out.append((r0.value, n.value))
    return out


class Multi:
    """One scenario on a row-partitioned domain (the paper's per-core strips
    with halo exchange every RK stage), through the C ABI."""

    def __init__(self, sc, nparts: int, precision: int = F32, stream: Optional[int] = None, tile: int = 0):
        self.sc = sc
        self.nx, self.ny = sc.nx, sc.ny
        self._m = ctypes.c_void_p()
        b = np.ascontiguousarray(sc.b, dtype=np.float64)
        self.params = params_for(sc, precision, stream, tile)
        _check(lib.swe_multi_create(ctypes.byref(Grid(sc.nx, sc.ny)), float(sc.dx), float(sc.dy), _dp(b),
                                    ctypes.byref(self.params), int(nparts), ctypes.byref(self._m)), "swe_multi_create")
        if sc.t0:
            _check(lib.swe_multi_set_time(self._m, float(sc.t0)), "swe_multi_set_time")
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (sc.h, sc.hu, sc.hv)]
        _check(lib.swe_multi_set_state(self._m, *[_dp(x) for x in a]), "swe_multi_set_state")

    def close(self) -> None:
        if self._m:
            lib.swe_multi_destroy(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n: int, cfl: Optional[float] = None) -> None:
        c = self.sc.cfl if cfl is None else cfl
        _check(lib.swe_multi_step(self._m, int(n), float(c)), "swe_multi_step")

    def get_state(self):
        out = tuple(np.empty((self.ny, self.nx), dtype=np.float64) for _ in range(3))
        _check(lib.swe_multi_get_state(self._m, *[_dp(x) for x in out]), "swe_multi_get_state")
        return out

    def mass(self) -> float:
        m = ctypes.c_double()
        _check(lib.swe_multi_mass(self._m, ctypes.byref(m)), "swe_multi_mass")
        return m.value

    def diagnostics(self, check: bool = True) -> Dict[str, float]:
        d = Diag()
        rc = lib.swe_multi_diagnostics(self._m, ctypes.byref(d))
        if check:
            _check(rc, "swe_multi_diagnostics")
        return _diag_dict(d)


def slot_bytes(nx: int, ny: int) -> int:
    """Device bytes one batch admission of an nx x ny grid takes."""
    return int(lib.swe_batch_slot_bytes(ctypes.byref(Grid(nx, ny))))


class Batch:
    """Independent scenarios advanced together by one persistent launch per
    run (the ensemble and serving path, FP32)."""

    def __init__(self, nslots: int, budget_bytes: int, template, stream: Optional[int] = None, tile: int = 0,
                 precision: int = F32):
        self._b = ctypes.c_void_p()
        self.nslots = int(nslots)
        self.params = params_for(template, precision, stream, tile)
        _check(lib.swe_batch_create(self.nslots, int(budget_bytes), ctypes.byref(self.params), ctypes.byref(self._b)),
               "swe_batch_create")
        self.shapes: Dict[int, Tuple[int, int]] = {}

    def close(self) -> None:
        if self._b:
            lib.swe_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def admit(self, sc, t_end: Optional[float] = None) -> int:
        """Admit a scenario; raises SweError (EBUDGET / EFULL) if it does not fit."""
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (sc.b, sc.h, sc.hu, sc.hv)]
        slot = ctypes.c_int32(-1)
        te = sc.t_end if t_end is None else t_end
        _check(lib.swe_batch_admit(self._b, ctypes.byref(Grid(sc.nx, sc.ny)), float(sc.dx), float(sc.dy),
                                   *[_dp(a) for a in arrs], float(te), ctypes.byref(slot)), "swe_batch_admit")
        self.shapes[slot.value] = (sc.ny, sc.nx)
        if getattr(sc, "t0", 0.0):
            _check(lib.swe_batch_set_time(self._b, slot.value, float(sc.t0)), "swe_batch_set_time")
        return slot.value

    def select(self, slots=None) -> None:
        """Advance only these live slots in the following runs (None: all)."""
        if slots is None:
            _check(lib.swe_batch_select(self._b, None, 0), "swe_batch_select")
            return
        arr = (ctypes.c_int32 * len(slots))(*[int(x) for x in slots])
        _check(lib.swe_batch_select(self._b, arr, len(slots)), "swe_batch_select")

    def times(self) -> np.ndarray:
        """Simulated time of every slot (NaN for free slots)."""
        t = np.empty(self.nslots, dtype=np.float64)
        _check(lib.swe_batch_times(self._b, _dp(t)), "swe_batch_times")
        return t

    def try_admit(self, sc, t_end: Optional[float] = None) -> Optional[int]:
        """admit, or None when the scenario does not fit now (budget, slots or
        device memory: the batch is unchanged and a later try may succeed)."""
        try:
            return self.admit(sc, t_end)
        except SweError as e:
            if e.code in (EBUDGET, EFULL, ENOMEM):
                return None
            raise

    def run(self, k: int, cfl: float = 0.4) -> None:
        _check(lib.swe_batch_run(self._b, int(k), float(cfl)), "swe_batch_run")

    def poll(self):
        out = (ctypes.c_int32 * self.nslots)()
        n = ctypes.c_int32()
        _check(lib.swe_batch_poll(self._b, out, ctypes.byref(n)), "swe_batch_poll")
        return [out[k] for k in range(n.value)]

    def status(self) -> int:
        return int(lib.swe_batch_status(self._b))

    def check_word(self, slot: int) -> int:
        """Checked build: the slot's first out-of-range index recorded (0: none)."""
        w = ctypes.c_uint64()
        _check(lib.swe_batch_check_status(self._b, int(slot), ctypes.byref(w)), "swe_batch_check_status")
        return int(w.value)

    def get_state(self, slot: int):
        ny, nx = self.shapes[slot]
        out = tuple(np.empty((ny, nx)) for _ in range(3))
        _check(lib.swe_batch_get_state(self._b, int(slot), *[_dp(x) for x in out]), "swe_batch_get_state")
        return out

    def diagnostics(self, slot: int, check: bool = True) -> Dict[str, float]:
        d = Diag()
        rc = lib.swe_batch_diagnostics(self._b, int(slot), ctypes.byref(d))
        if check:
            _check(rc, "swe_batch_diagnostics")
        return _diag_dict(d)

    def retire(self, slot: int, want_state: bool = True):
        ny, nx = self.shapes[slot]
        st = tuple(np.empty((ny, nx)) for _ in range(3)) if want_state else None
        m, r = ctypes.c_double(), ctypes.c_double()
        ptrs = [_dp(x) for x in st] if st else [None, None, None]
        _check(lib.swe_batch_retire(self._b, int(slot), *ptrs, ctypes.byref(m), ctypes.byref(r)), "swe_batch_retire")
        del self.shapes[slot]
        return st, m.value, r.value

    def memory(self) -> Tuple[int, int]:
        u, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib.swe_batch_memory(self._b, ctypes.byref(u), ctypes.byref(b)), "swe_batch_memory")
        return u.value, b.value

    def set_barrier(self, timeout_s: float, extra_arrivals: int = 0) -> None:
        _check(lib.swe_batch_set_barrier(self._b, float(timeout_s), int(extra_arrivals)), "swe_batch_set_barrier")
