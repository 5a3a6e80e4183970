"""ctypes binding of the C oracle (test infrastructure only).

Wraps the plain C restatement of 2D-PT (Algorithm 1) in ``pt2d_oracle.c``:
Philox4x32-10, pt_exp, the heat-bath decision, the swap test, the energies of
Eq. 1 and the full 2D-PT loop over a chosen subset of independent runs.
"""
from __future__ import annotations

import contextlib
import ctypes as C

import numpy as np

from . import _build
from .coloring import greedy_color
from .sparsify import PhysInstance

_lib = None


def load(path: str):
    """Load and configure an oracle shared library at `path`."""
    L = C.CDLL(path)
    L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    L.orc_philox4x32_10.restype = None
    L.orc_pt_exp.argtypes = [C.c_float]
    L.orc_pt_exp.restype = C.c_float
    L.orc_heatbath.argtypes = [C.c_float, C.c_int32, C.c_uint32]
    L.orc_heatbath.restype = C.c_int
    L.orc_swap_accept.argtypes = [C.c_float, C.c_uint32]
    L.orc_swap_accept.restype = C.c_int
    L.orc_cost_f.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_cost_f.restype = C.c_int64
    L.orc_constraint_g.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_constraint_g.restype = C.c_int64
    L.orc_local_field.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]
    L.orc_local_field.restype = C.c_int32
    L.orc_init_walker.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, C.c_int32, C.c_void_p]
    L.orc_init_walker.restype = None
    L.orc_sweep_walker.argtypes = [C.c_void_p, C.c_uint64, C.c_int32, C.c_int32, C.c_int64,
                                   C.c_float, C.c_int32, C.c_void_p]
    L.orc_sweep_walker.restype = None
    L.orc_pt2d_run.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                               C.c_int32, C.c_void_p, C.c_uint64, C.c_int64, C.c_int32,
                               C.c_void_p]
    L.orc_pt2d_run.restype = C.c_int
    L.orc_heatbath_count.argtypes = [C.c_float, C.c_int32]
    L.orc_heatbath_count.restype = C.c_int64
    L.orc_swap_count.argtypes = [C.c_float]
    L.orc_swap_count.restype = C.c_int64
    L.orc_pt_exp_constants.argtypes = [C.POINTER(C.c_float)]
    L.orc_pt_exp_constants.restype = None
    L.orc_swap_event.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32, C.c_int64,
                                 C.c_int, C.c_void_p, C.c_void_p]
    L.orc_swap_event.restype = None
    for name in ("orc_pt_exp_array", "orc_swap_accept_array", "orc_philox_array"):
        getattr(L, name).restype = None
    L.orc_pt_exp_array.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.orc_heatbath_array.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.orc_heatbath_array.restype = None
    L.orc_swap_accept_array.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.orc_philox_array.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call to another build (mutation tests)."""
    global _lib
    saved = _lib
    _lib = load(path)
    try:
        yield _lib
    finally:
        _lib = saved


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _OrcInst(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("cp_ptr", C.c_void_p),
        ("cp_col", C.c_void_p),
        ("cp_J", C.c_void_p),
        ("lk_ptr", C.c_void_p),
        ("lk_col", C.c_void_p),
        ("h", C.c_void_p),
        ("color", C.c_void_p),
        ("n_colors", C.c_int32),
        ("lk_w", C.c_void_p),
        ("hk", C.c_void_p),
        ("g0", C.c_int64),
    ]


class _OrcState(C.Structure):
    _fields_ = [
        ("spins", C.c_void_p),
        ("walker_at", C.c_void_p),
        ("f", C.c_void_p),
        ("g", C.c_void_p),
        ("counters", C.c_void_p),
        ("trace_cap", C.c_int64),
        ("trace_f", C.c_void_p),
        ("trace_g", C.c_void_p),
        ("best_f", C.c_void_p),
        ("best_event", C.c_void_p),
        ("best_state", C.c_void_p),
        ("target", C.c_void_p),
        ("solved_event", C.c_void_p),
        ("acc_P", C.c_void_p),
        ("acc_B", C.c_void_p),
        ("hist", C.c_void_p),
        ("hist_slot", C.c_int64),
        ("sum_f", C.c_void_p),
        ("sum_g", C.c_void_p),
        ("n_feasible", C.c_void_p),
        ("mode", C.c_int64),
    ]


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def pt_exp(x: float) -> float:
    return float(np.float32(lib().orc_pt_exp(float(np.float32(x)))))


def heatbath(beta: float, H: int, r: int) -> int:
    return int(lib().orc_heatbath(float(np.float32(beta)), int(H), int(r) & 0xFFFFFFFF))


def swap_accept(x: float, r: int) -> int:
    return int(lib().orc_swap_accept(float(np.float32(x)), int(r) & 0xFFFFFFFF))


def heatbath_count(beta: float, H: int) -> int:
    return int(lib().orc_heatbath_count(float(np.float32(beta)), int(H)))


def swap_count(x: float) -> int:
    return int(lib().orc_swap_count(float(np.float32(x))))


def pt_exp_constants() -> np.ndarray:
    out = (C.c_float * 11)()
    lib().orc_pt_exp_constants(out)
    return np.array(list(out), dtype=np.float32)


def pt_exp_array(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_pt_exp_array(_p(x), _p(y), x.size)
    return y


def heatbath_array(beta, H, r) -> np.ndarray:
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.empty(beta.size, dtype=np.int8)
    lib().orc_heatbath_array(_p(beta), _p(H), _p(r), _p(out), beta.size)
    return out


def swap_accept_array(x, r) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.empty(x.size, dtype=np.int8)
    lib().orc_swap_accept_array(_p(x), _p(r), _p(out), x.size)
    return out


def philox_array(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().orc_philox_array(_p(ctr), _p(key), _p(out), ctr.shape[0])
    return out


def swap_event(beta, P, f_w, g_w, walker_at, seed: int, run: int, event: int, direction: int):
    """One swap event of Algorithm 1 on one run's slot->walker map (copied);
    returns (walker_at, acc_P, acc_B)."""
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.int32)
    f_w = np.ascontiguousarray(f_w, dtype=np.int64)
    g_w = np.ascontiguousarray(g_w, dtype=np.int64)
    at = np.array(walker_at, dtype=np.int32, copy=True)
    accP = np.zeros(at.size, np.int64)
    accB = np.zeros(at.size, np.int64)
    lib().orc_swap_event(beta.size, _p(beta), P.size, _p(P), _p(f_w), _p(g_w), _p(at), int(seed),
                         int(run), int(event), int(direction), _p(accP), _p(accB))
    return at, accP, accB


class OracleInstance:
    """A physical instance plus its greedy colouring, pinned in C-compatible arrays."""

    def __init__(self, inst: PhysInstance, color: np.ndarray | None = None):
        self.inst = inst
        self.n = inst.n
        self.cp_ptr = np.ascontiguousarray(inst.cp_ptr, dtype=np.int32)
        self.cp_col = np.ascontiguousarray(inst.cp_col, dtype=np.int32)
        self.cp_J = np.ascontiguousarray(inst.cp_J, dtype=np.int16)
        self.lk_ptr = np.ascontiguousarray(inst.lk_ptr, dtype=np.int32)
        self.lk_col = np.ascontiguousarray(inst.lk_col, dtype=np.int32)
        self.h = None if inst.h is None else np.ascontiguousarray(inst.h, dtype=np.int32)
        lk_w, hk = getattr(inst, "lk_w", None), getattr(inst, "hk", None)
        self.lk_w = None if lk_w is None else np.ascontiguousarray(lk_w, dtype=np.int16)
        self.hk = None if hk is None else np.ascontiguousarray(hk, dtype=np.int32)
        self.g0 = int(getattr(inst, "g0", 0))
        if color is None:
            color, n_colors = greedy_color(inst.n, self.cp_ptr, self.cp_col, self.lk_ptr, self.lk_col)
        else:
            color = np.asarray(color, dtype=np.int32)
            n_colors = int(color.max()) + 1
        self.color = np.ascontiguousarray(color, dtype=np.int32)
        self.n_colors = n_colors
        self._c = _OrcInst(self.n, _p(self.cp_ptr), _p(self.cp_col), _p(self.cp_J), _p(self.lk_ptr),
                           _p(self.lk_col), _p(self.h), _p(self.color), self.n_colors,
                           _p(self.lk_w), _p(self.hk), self.g0)

    @property
    def ref(self):
        return C.byref(self._c)

    def cost_f(self, s: np.ndarray) -> int:
        s = np.ascontiguousarray(s, dtype=np.int8)
        return int(lib().orc_cost_f(self.ref, _p(s)))

    def constraint_g(self, s: np.ndarray) -> int:
        s = np.ascontiguousarray(s, dtype=np.int8)
        return int(lib().orc_constraint_g(self.ref, _p(s)))

    def local_field(self, s: np.ndarray, a: int, P: int) -> int:
        s = np.ascontiguousarray(s, dtype=np.int8)
        return int(lib().orc_local_field(self.ref, _p(s), int(a), int(P)))

    def init_walker(self, seed: int, run: int, walker: int) -> np.ndarray:
        s = np.zeros(self.n, dtype=np.int8)
        lib().orc_init_walker(self.ref, int(seed), int(run), int(walker), _p(s))
        return s

    def sweep_walker(self, s: np.ndarray, seed: int, run: int, walker: int, sweep_index: int,
                     beta: float, P: int) -> None:
        assert s.dtype == np.int8 and s.flags.c_contiguous
        lib().orc_sweep_walker(self.ref, int(seed), int(run), int(walker), int(sweep_index),
                               float(np.float32(beta)), int(P), _p(s))


class OracleRun:
    """State of a set of independent 2D-PT runs (Algorithm 1) on one instance."""

    def __init__(self, oinst: OracleInstance, beta, P, run_ids, seed: int, trace_cap: int = 0,
                 target=None, hist: bool = False, hist_slot: int = -1, mode: int = 0):
        """mode 0: 2D-PT (Algorithm 1).  mode 1: the J-column PT baseline -- every
        event is a beta-swap event (odd / even pairs alternating), so replicas
        never change column, and each event records the last row's replica of
        lowest g, then lowest f, then lowest column."""
        self.oinst = oinst
        self.beta = np.ascontiguousarray(beta, dtype=np.float32)
        self.P = np.ascontiguousarray(P, dtype=np.int32)
        self.I = int(self.beta.size)
        self.J = int(self.P.size)
        self.R = self.I * self.J
        self.run_ids = np.ascontiguousarray(run_ids, dtype=np.int32)
        self.n_runs = int(self.run_ids.size)
        self.seed = int(seed)
        n, R, q = oinst.n, self.R, self.n_runs
        self.spins = np.zeros((q, R, n), dtype=np.int8)
        self.walker_at = np.zeros((q, R), dtype=np.int32)
        self.f = np.zeros((q, R), dtype=np.int64)
        self.g = np.zeros((q, R), dtype=np.int64)
        self.counters = np.zeros(4, dtype=np.int64)
        self.trace_cap = int(trace_cap)
        self.trace_f = np.zeros((q, max(trace_cap, 1)), dtype=np.int64) if trace_cap else None
        self.trace_g = np.zeros((q, max(trace_cap, 1)), dtype=np.int64) if trace_cap else None
        self.best_f = np.zeros(q, dtype=np.int64)
        self.best_event = np.zeros(q, dtype=np.int64)
        self.best_state = np.zeros((q, n), dtype=np.int8)
        self.target = None if target is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(target, dtype=np.int64), (q,)))
        self.solved_event = np.zeros(q, dtype=np.int64)
        self.acc_P = np.zeros((q, R), dtype=np.int64)
        self.acc_B = np.zeros((q, R), dtype=np.int64)
        self.hist_slot = int(hist_slot)
        if hist:
            if n > 24:
                raise ValueError("histograms need n <= 24")
            shape = (q, R, 1 << n) if hist_slot < 0 else (q, 1 << n)
            self.hist = np.zeros(shape, dtype=np.uint32)
        else:
            self.hist = None
        self.sum_f = np.zeros((q, R), dtype=np.int64)
        self.sum_g = np.zeros((q, R), dtype=np.int64)
        self.n_feasible = np.zeros((q, R), dtype=np.int64)
        self._st = _OrcState(_p(self.spins), _p(self.walker_at), _p(self.f), _p(self.g),
                             _p(self.counters), self.trace_cap, _p(self.trace_f), _p(self.trace_g),
                             _p(self.best_f), _p(self.best_event), _p(self.best_state),
                             _p(self.target), _p(self.solved_event), _p(self.acc_P), _p(self.acc_B),
                             _p(self.hist), self.hist_slot, _p(self.sum_f), _p(self.sum_g),
                             _p(self.n_feasible), int(mode))

    def run(self, sweeps: int, interval: int) -> None:
        rc = lib().orc_pt2d_run(self.oinst.ref, self.I, _p(self.beta), self.J, _p(self.P),
                                self.n_runs, _p(self.run_ids), self.seed, int(sweeps), int(interval),
                                C.byref(self._st))
        if rc != 0:
            raise ValueError(f"orc_pt2d_run failed ({rc})")

    @property
    def sweeps_done(self) -> int:
        return int(self.counters[0])

    @property
    def events_done(self) -> int:
        return int(self.counters[1])

    def slot_of(self) -> np.ndarray:
        """Inverse permutation: walker -> slot."""
        out = np.empty_like(self.walker_at)
        for q in range(self.n_runs):
            out[q, self.walker_at[q]] = np.arange(self.R, dtype=np.int32)
        return out
