"""Plain FP64 CPU oracle for the improved ETD particle method.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1404_1160_gb300`` and the library never
imports it.

The arithmetic lives in ``oracle.c`` (scalar C, FP64, compiled with
floating-point contraction off).  This module only builds and loads it and
marshals numpy arrays.  Each wrapper names the passage of Frenod, Hirstoaga &
Lutz that the C function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from dataclasses import field as _dc_field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELD_POISSON, FIELD_DUFFING, FIELD_ZERO = 0, 1, 2
FINE_RK4, FINE_LAWSON = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = [
        "gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
        "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("eps", C.c_double),
        ("dt", C.c_double),
        ("field_model", C.c_int32),
        ("fine_solver", C.c_int32),
        ("steps_per_turn", C.c_int32),
        ("n_cells", C.c_int32),
        ("r_min", C.c_double),
        ("r_max", C.c_double),
        ("total_charge", C.c_double),
        ("weight_fixed", C.c_uint64),
        ("max_window_steps", C.c_int32),
        ("field_parity", C.c_int32),
    ]


class Derived(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("h", "inv_eps", "D", "ch", "sh", "c1", "s1", "hr", "inv_hr", "q_unit")]


class StepStats(C.Structure):
    _fields_ = [
        ("window_steps", C.c_int64),
        ("n_no_period", C.c_int64),
        ("T_min", C.c_double),
        ("T_max", C.c_double),
        ("T_mean", C.c_double),
        ("N_min", C.c_int64),
        ("N_max", C.c_int64),
    ]


@dataclass
class Config:
    """Problem statement of the paper (Sec. 1, 2.1, 2.3, Remark 3.4)."""

    eps: float = 0.01
    dt: float = 0.1
    field_model: int = FIELD_POISSON
    fine_solver: int = FINE_LAWSON
    steps_per_turn: int = 100
    n_cells: int = 256
    r_min: float = -4.0
    r_max: float = 4.0
    total_charge: float = 1.0
    weight_fixed: int = 1 << 32
    max_window_steps: int = 300
    field_parity: int = 0  # 0: E = (1/r) int_0^r rho (even); 1: its odd extension

    def to_c(self) -> Params:
        return Params(
            self.eps, self.dt, self.field_model, self.fine_solver, self.steps_per_turn,
            self.n_cells, self.r_min, self.r_max, self.total_charge, self.weight_fixed,
            self.max_window_steps, self.field_parity,
        )


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            P = C.POINTER
            d, i64, i32 = C.c_double, C.c_int64, C.c_int
            pd, pi64 = P(d), P(i64)
            sig = {
                "orc_derive": (i32, [P(Params), P(Derived)]),
                "orc_deposit": (i32, [P(Params), i64, pd, pi64, pi64]),
                "orc_deposit_f32": (i32, [P(Params), i64, P(C.c_float), pi64, pi64]),
                "orc_classic_step": (i32, [P(Params), i64, pd, pd, i32, pd]),
                "orc_poisson": (i32, [P(Params), i64, pi64, pi64, pd, pd]),
                "orc_gather": (i32, [P(Params), i64, pd, pd, pd, pd]),
                "orc_field": (i32, [P(Params), i64, pd, pd]),
                "orc_fine_steps": (i32, [P(Params), i64, pd, pd, d, i64]),
                "orc_brute_force": (i32, [P(Params), i64, pd, pd, d]),
                "orc_periods": (i32, [P(Params), i64, pd, pd, pd, pi64, pi64]),
                "orc_etd_step": (i32, [P(Params), i64, pd, pd, pd, i32, pi64, pd, P(StepStats)]),
                "orc_quad_root": (d, [d, d, d]),
                "orc_interp": (d, [d, d, d, d]),
                "orc_duffing_b2": (d, [d, d, d]),
                "orc_duffing_period_agm": (d, [d, d, d]),
                "orc_duffing_period_quad": (d, [d, d, d, i32]),
                "orc_duffing_period_series": (d, [d, d, d]),
                "orc_duffing_energy": (d, [d, d, d]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def derive(cfg: Config) -> Derived:
    d = Derived()
    _check(_load().orc_derive(C.byref(cfg.to_c()), C.byref(d)), "derive")
    return d


def deposit(cfg: Config, R):
    """CIC deposit in W-unit integers (Sec. 2.3).  Returns (Q, n_out)."""
    R = _f64(R)
    Q = np.zeros(cfg.n_cells + 1, np.int64)
    n_out = np.zeros(1, np.int64)
    _check(_load().orc_deposit(C.byref(cfg.to_c()), R.size, _pd(R), _pi64(Q), _pi64(n_out)), "deposit")
    return Q, int(n_out[0])


def deposit_f32(cfg: Config, R):
    """The CIC deposit with binary32 position arithmetic (the FP32 form's quantisation)."""
    R = np.ascontiguousarray(R, dtype=np.float32)
    Q = np.zeros(cfg.n_cells + 1, np.int64)
    n_out = np.zeros(1, np.int64)
    _check(_load().orc_deposit_f32(C.byref(cfg.to_c()), R.size, R.ctypes.data_as(C.POINTER(C.c_float)), _pi64(Q),
                                   _pi64(n_out)), "deposit_f32")
    return Q, int(n_out[0])


def poisson(cfg: Config, Q, n_particles: int):
    """Trapezoid integral of d/dr(rE) = rho (eq. VlasPoissAxSymBeam).  Returns (S, E, rE_edges)."""
    Q = np.ascontiguousarray(Q, np.int64)
    S = np.zeros(cfg.n_cells + 1, np.int64)
    E = np.zeros(cfg.n_cells + 1, np.float64)
    edges = np.zeros(2, np.float64)
    _check(_load().orc_poisson(C.byref(cfg.to_c()), n_particles, _pi64(Q), _pi64(S), _pd(E), _pd(edges)), "poisson")
    return S, E, edges


def gather(cfg: Config, R, E, edges):
    """Linear interpolation of the mesh field at the particles (Sec. 2.3)."""
    R, E, edges = _f64(R), _f64(E), _f64(edges)
    out = np.zeros(R.size, np.float64)
    _check(_load().orc_gather(C.byref(cfg.to_c()), R.size, _pd(R), _pd(E), _pd(edges), _pd(out)), "gather")
    return out


def field(cfg: Config, R):
    """E at every particle for the configured field model."""
    R = _f64(R)
    out = np.zeros(R.size, np.float64)
    _check(_load().orc_field(C.byref(cfg.to_c()), R.size, _pd(R), _pd(out)), "field")
    return out


def fine_steps(cfg: Config, R, V, n_fine: int, h_step: float | None = None):
    """n_fine fine steps of the whole particle system (RK4 or Lawson RK4)."""
    R, V = _f64(R).copy(), _f64(V).copy()
    h = derive(cfg).h if h_step is None else h_step
    _check(_load().orc_fine_steps(C.byref(cfg.to_c()), R.size, _pd(R), _pd(V), h, n_fine), "fine_steps")
    return R, V


def brute_force(cfg: Config, R, V, t: float):
    """The paper's reference solution: fine steps of 2*pi*eps/S up to time t."""
    R, V = _f64(R).copy(), _f64(V).copy()
    _check(_load().orc_brute_force(C.byref(cfg.to_c()), R.size, _pd(R), _pd(V), t), "brute_force")
    return R, V


def periods(cfg: Config, R, V):
    """Step 1 of Algorithm ETDFSSModAlgo (Remark CompOfThePeriodsRem): T in fine steps."""
    R, V = _f64(R), _f64(V)
    T = np.zeros(R.size, np.float64)
    nf = np.zeros(1, np.int64)
    K = np.zeros(1, np.int64)
    _check(_load().orc_periods(C.byref(cfg.to_c()), R.size, _pd(R), _pd(V), _pd(T), _pi64(nf), _pi64(K)), "periods")
    return T, int(nf[0]), int(K[0])


@dataclass
class StepResult:
    R: np.ndarray
    V: np.ndarray
    T: np.ndarray
    N: np.ndarray
    o: np.ndarray
    stats: dict = _dc_field(default_factory=dict)


def etd_step(cfg: Config, R, V, T=None) -> StepResult:
    """One macro step of Algorithm ETDFSSModAlgo.  T (fine steps) known => step 1 skipped."""
    R, V = _f64(R).copy(), _f64(V).copy()
    known = T is not None
    Tarr = _f64(T).copy() if known else np.zeros(R.size, np.float64)
    N = np.zeros(R.size, np.int64)
    o = np.zeros(R.size, np.float64)
    st = StepStats()
    _check(
        _load().orc_etd_step(C.byref(cfg.to_c()), R.size, _pd(R), _pd(V), _pd(Tarr), int(known), _pi64(N), _pd(o), C.byref(st)),
        "etd_step",
    )
    stats = {k: getattr(st, k) for k, _ in StepStats._fields_}
    return StepResult(R, V, Tarr, N, o, stats)


def classic_step(cfg: Config, R, V, mode: int):
    """One macro step of Algorithm ClassicETDAlgo: mode 0 with P = 2 pi eps, mode 1
    (modified ETD) with P = the mean first-tour time.  Returns (R, V, P)."""
    R, V = _f64(R).copy(), _f64(V).copy()
    P = np.zeros(1, np.float64)
    _check(_load().orc_classic_step(C.byref(cfg.to_c()), R.size, _pd(R), _pd(V), int(mode), _pd(P)), "classic_step")
    return R, V, float(P[0])


def quad_root(v0, v1, v2) -> float:
    return _load().orc_quad_root(v0, v1, v2)


def interp(y0, y1, y2, s) -> float:
    return _load().orc_interp(y0, y1, y2, s)


def duffing_b2(eps, r0, v0) -> float:
    return _load().orc_duffing_b2(eps, r0, v0)


def duffing_period_agm(eps, r0, v0) -> float:
    return _load().orc_duffing_period_agm(eps, r0, v0)


def duffing_period_quad(eps, r0, v0, n_nodes=64) -> float:
    return _load().orc_duffing_period_quad(eps, r0, v0, n_nodes)


def duffing_period_series(eps, r0, v0) -> float:
    return _load().orc_duffing_period_series(eps, r0, v0)


def duffing_energy(eps, r, v) -> float:
    return _load().orc_duffing_energy(eps, r, v)
