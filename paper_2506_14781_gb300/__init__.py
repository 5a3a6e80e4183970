"""GB300-native two-dimensional parallel tempering (arxiv 2506.14781).

Python face of the C ABI in include/pt2d.h.  Every step of the method runs in
the CUDA library libpt2d.so; this module only marshals arguments.  PyTorch,
when used, only provides device memory (the context workspace) and the CUDA
stream.  Importing works without a GPU; creating a context needs one.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import _lib
from ._lib import (ACC_B, ACC_P, BEST_EVENT, BEST_F, BEST_STATE, COLORS, COUNTERS, F, G,
                   N_FEASIBLE, SOLVED_EVENT, STATES, SUM_F, SUM_G, TARGET, TRACE_F, TRACE_G,
                   WALKER_AT, Pt2dError)

__all__ = [
    "PhysicalInstance", "sparsify", "greedy_color", "plan_tiling", "PT2D", "Batch", "PoolFull", "Server",
    "Pt2dError", "onehot_penalty", "equality_penalty", "adaptive_schedule",
    "diag_philox",
    "diag_pt_exp", "diag_heatbath", "diag_swap_accept", "diag_read_bandwidth", "STATES", "WALKER_AT", "F", "G",
    "COUNTERS", "TRACE_F", "TRACE_G", "BEST_F", "BEST_EVENT", "BEST_STATE", "SOLVED_EVENT",
    "ACC_P", "ACC_B", "SUM_F", "SUM_G", "N_FEASIBLE", "COLORS", "TARGET",
]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


@dataclasses.dataclass
class PhysicalInstance:
    """Sparsified (physical) constrained Ising instance: symmetric coupling CSR
    with int16 values and symmetric copy-link CSR (see pt2d_instance)."""
    n: int
    cp_ptr: np.ndarray
    cp_col: np.ndarray
    cp_J: np.ndarray
    lk_ptr: np.ndarray
    lk_col: np.ndarray
    h: np.ndarray | None = None
    color: np.ndarray | None = None
    copy_of: np.ndarray | None = None
    lk_w: np.ndarray | None = None   # int16 penalty weight K of each link entry (None: 1)
    hk: np.ndarray | None = None     # int32 penalty field k (None: 0)
    g0: int = 0                      # constant term of g

    def __post_init__(self):
        self.cp_ptr = np.ascontiguousarray(self.cp_ptr, dtype=np.int32)
        self.cp_col = np.ascontiguousarray(self.cp_col, dtype=np.int32)
        self.cp_J = np.ascontiguousarray(self.cp_J, dtype=np.int16)
        self.lk_ptr = np.ascontiguousarray(self.lk_ptr, dtype=np.int32)
        self.lk_col = np.ascontiguousarray(self.lk_col, dtype=np.int32)
        if self.h is not None:
            self.h = np.ascontiguousarray(self.h, dtype=np.int32)
        if self.color is not None:
            self.color = np.ascontiguousarray(self.color, dtype=np.int32)
        if self.lk_w is not None:
            self.lk_w = np.ascontiguousarray(self.lk_w, dtype=np.int16)
        if self.hk is not None:
            self.hk = np.ascontiguousarray(self.hk, dtype=np.int32)

    def c_struct(self) -> _lib.Instance:
        return _lib.Instance(int(self.n), _p(self.cp_ptr), _p(self.cp_col), _p(self.cp_J),
                             _p(self.lk_ptr), _p(self.lk_col), _p(self.h), _p(self.color),
                             _p(self.lk_w), _p(self.hk), int(self.g0))


_RULES = {"fixed": _lib.SPARSIFY_FIXED, "max_edges": _lib.SPARSIFY_MAX_EDGES,
          "max_degree": _lib.SPARSIFY_MAX_DEGREE}


def sparsify(Jq: np.ndarray, rule: str, param: int) -> PhysicalInstance:
    """Copy-chain sparsification (pt2d_sparsify) of a dense int16 logical matrix."""
    Jq = np.ascontiguousarray(Jq, dtype=np.int16)
    N = Jq.shape[0]
    L = _lib.lib()
    n = C.c_int32()
    ncp = C.c_int64()
    nlk = C.c_int64()
    st = L.pt2d_sparsify(N, _p(Jq), _RULES[rule], int(param), C.byref(n), C.byref(ncp),
                         C.byref(nlk), None, None, None, None, None, None)
    _lib.check(st, "pt2d_sparsify")
    cp_ptr = np.zeros(n.value + 1, np.int32)
    cp_col = np.zeros(max(ncp.value, 1), np.int32)
    cp_J = np.zeros(max(ncp.value, 1), np.int16)
    lk_ptr = np.zeros(n.value + 1, np.int32)
    lk_col = np.zeros(max(nlk.value, 1), np.int32)
    copy_of = np.zeros(n.value, np.int32)
    st = L.pt2d_sparsify(N, _p(Jq), _RULES[rule], int(param), C.byref(n), C.byref(ncp),
                         C.byref(nlk), _p(cp_ptr), _p(cp_col), _p(cp_J), _p(lk_ptr), _p(lk_col),
                         _p(copy_of))
    _lib.check(st, "pt2d_sparsify")
    return PhysicalInstance(n.value, cp_ptr, cp_col[:ncp.value], cp_J[:ncp.value], lk_ptr,
                            lk_col[:nlk.value], copy_of=copy_of)


def onehot_penalty(n: int, groups) -> tuple:
    """Penalty terms (lk_ptr, lk_col, lk_w, hk, g0) of one-hot constraints over
    `groups` (lists of spin ids): g = sum_c (sum_{a in c} [s_a = +1] - 1)^2
    (pt2d_onehot_penalty)."""
    grp_ptr = np.concatenate([[0], np.cumsum([len(g) for g in groups])]).astype(np.int32)
    grp_col = np.ascontiguousarray(np.concatenate([np.asarray(g, np.int32) for g in groups])
                                   if groups else np.zeros(0, np.int32), dtype=np.int32)
    L = _lib.lib()
    lk_ptr = np.zeros(n + 1, np.int32)
    hk = np.zeros(n, np.int32)
    nnz = C.c_int32()
    g0 = C.c_int64()
    L.pt2d_onehot_penalty(int(n), len(groups), _p(grp_ptr), _p(grp_col), _p(lk_ptr), None, None, 0,
                          C.byref(nnz), _p(hk), C.byref(g0))
    lk_col = np.zeros(max(nnz.value, 1), np.int32)
    lk_w = np.zeros(max(nnz.value, 1), np.int16)
    _lib.check(L.pt2d_onehot_penalty(int(n), len(groups), _p(grp_ptr), _p(grp_col), _p(lk_ptr),
                                     _p(lk_col), _p(lk_w), int(lk_col.size), C.byref(nnz), _p(hk),
                                     C.byref(g0)), "pt2d_onehot_penalty")
    return lk_ptr, lk_col[:nnz.value].copy(), lk_w[:nnz.value].copy(), hk, int(g0.value)


def equality_penalty(n: int, constraints) -> tuple:
    """Penalty terms (lk_ptr, lk_col, lk_w, hk, g0) of linear equality
    constraints: `constraints` is a list of (spin ids, integer coefficients,
    right-hand side b), g = sum_c (sum_a A_a [s_a = +1] - b_c)^2
    (pt2d_equality_penalty)."""
    con_ptr = np.concatenate([[0], np.cumsum([len(c[0]) for c in constraints])]).astype(np.int32)
    if constraints:
        con_col = np.ascontiguousarray(np.concatenate([np.asarray(c[0], np.int32) for c in constraints]),
                                       dtype=np.int32)
        coef = np.ascontiguousarray(np.concatenate([np.asarray(c[1], np.int64) for c in constraints]),
                                    dtype=np.int64)
        if coef.size and (coef.min() < -2 ** 31 or coef.max() >= 2 ** 31):
            raise ValueError("equality_penalty: coefficients must fit int32")
        coef = coef.astype(np.int32)
    else:
        con_col = np.zeros(0, np.int32)
        coef = np.zeros(0, np.int32)
    rhs = np.array([int(c[2]) for c in constraints], np.int64)
    L = _lib.lib()
    lk_ptr = np.zeros(n + 1, np.int32)
    hk = np.zeros(n, np.int32)
    nnz = C.c_int32()
    g0 = C.c_int64()
    args = (int(n), len(constraints), _p(con_ptr), _p(con_col), _p(coef), _p(rhs), _p(lk_ptr))
    L.pt2d_equality_penalty(*args, None, None, 0, C.byref(nnz), _p(hk), C.byref(g0))
    lk_col = np.zeros(max(nnz.value, 1), np.int32)
    lk_w = np.zeros(max(nnz.value, 1), np.int16)
    _lib.check(L.pt2d_equality_penalty(*args, _p(lk_col), _p(lk_w), int(lk_col.size), C.byref(nnz), _p(hk),
                                       C.byref(g0)), "pt2d_equality_penalty")
    return lk_ptr, lk_col[:nnz.value].copy(), lk_w[:nnz.value].copy(), hk, int(g0.value)


def greedy_color(inst: PhysicalInstance):
    """Greedy colouring (pt2d_greedy_color): (colour array, number of colours)."""
    color = np.zeros(inst.n, np.int32)
    nc = C.c_int32()
    cs = inst.c_struct()
    _lib.check(_lib.lib().pt2d_greedy_color(C.byref(cs), _p(color), C.byref(nc)),
               "pt2d_greedy_color")
    return color, nc.value


SWAP_MODES = {"2d": 0, "jcolumn": 1}


class PT2D:
    """One 2D-PT context: `runs` independent I x J replica grids on one instance.

    workspace: "library" (the library allocates device memory with cudaMalloc),
    or "torch" (a torch uint8 CUDA tensor owned by this object provides it).
    sweep_kernel: "auto", "global" (replica slab in global memory), "smem"
    (int8 slab held in shared memory for a whole swap interval) or "bits"
    (bit-packed slab in shared memory, for instances whose int8 slab does not fit).
    stream: a torch.cuda.Stream, a raw cudaStream_t (int), or None (default stream).
    swap_mode: "2d" (Algorithm 1) or "jcolumn" (the J-column PT baseline: beta-swaps
    only, so each column is a standard PT; events record the best last-row replica).
    """

    def __init__(self, inst: PhysicalInstance, beta, P, runs: int, *, stream=None,
                 workspace: str = "library", trace_capacity: int = 1024,
                 walkers_per_cta: int = 0, threads_per_cta: int = 0, device: int = -1,
                 profile: bool = False, sweep_kernel: str = "auto",
                 walkers_per_thread: int = 0, swap_mode: str = "2d"):
        self.inst = inst
        self.beta = np.ascontiguousarray(beta, dtype=np.float32)
        self.P = np.ascontiguousarray(P, dtype=np.int32)
        self.I, self.J = int(self.beta.size), int(self.P.size)
        self.R = self.I * self.J
        self.runs = int(runs)
        self.n = int(inst.n)
        self.trace_capacity = int(trace_capacity)
        L = _lib.lib()
        opt = _lib.Options()
        L.pt2d_default_options(C.byref(opt))
        opt.trace_capacity = int(trace_capacity)
        opt.walkers_per_cta = int(walkers_per_cta)
        opt.threads_per_cta = int(threads_per_cta)
        opt.device = int(device)
        opt.profile = 1 if profile else 0
        opt.sweep_kernel = {"auto": 0, "global": 1, "smem": 2, "bits": 3}[sweep_kernel]
        opt.walkers_per_thread = int(walkers_per_thread)
        opt.swap_mode = SWAP_MODES[swap_mode]
        self._stream_obj = stream
        if stream is not None:
            opt.stream = int(getattr(stream, "cuda_stream", stream))
        self._cs = inst.c_struct()
        self._ws = None
        if workspace == "torch":
            import torch

            need = C.c_size_t()
            _lib.check(L.pt2d_workspace_size(C.byref(self._cs), self.I, self.J, self.runs,
                                             C.byref(opt), C.byref(need)), "pt2d_workspace_size")
            dev = torch.device("cuda", device if device >= 0 else torch.cuda.current_device())
            self._ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
            opt.workspace = self._ws.data_ptr()
            opt.workspace_bytes = need.value
        elif workspace != "library":
            raise ValueError("workspace must be 'library' or 'torch'")
        self._ctx = C.c_void_p()
        st = L.pt2d_create(C.byref(self._ctx), C.byref(self._cs), self.I, _p(self.beta), self.J,
                           _p(self.P), self.runs, C.byref(opt))
        _lib.check(st, "pt2d_create")

    # shapes and dtypes of the readable arrays
    def _spec(self, what):
        q, R, n, T = self.runs, self.R, self.n, self.trace_capacity
        return {
            STATES: ((q, R, n), np.int8), WALKER_AT: ((q, R), np.int32), F: ((q, R), np.int64),
            G: ((q, R), np.int64), COUNTERS: ((4,), np.int64), TRACE_F: ((q, T), np.int64),
            TRACE_G: ((q, T), np.int64), BEST_F: ((q,), np.int64), BEST_EVENT: ((q,), np.int64),
            BEST_STATE: ((q, n), np.int8), SOLVED_EVENT: ((q,), np.int64),
            ACC_P: ((q, R), np.int64), ACC_B: ((q, R), np.int64), SUM_F: ((q, R), np.int64),
            SUM_G: ((q, R), np.int64), N_FEASIBLE: ((q, R), np.int64), COLORS: ((n,), np.int32),
            TARGET: ((q,), np.int64),
        }[what]

    def run(self, sweeps: int, swap_interval: int, seed: int) -> None:
        _lib.check(_lib.lib().pt2d_run(self._ctx, int(sweeps), int(swap_interval), int(seed)),
                   "pt2d_run", self._ctx)

    def read(self, what: int) -> np.ndarray:
        shape, dt = self._spec(what)
        out = np.empty(shape, dtype=dt)
        _lib.check(_lib.lib().pt2d_read(self._ctx, what, _p(out), out.nbytes), "pt2d_read",
                   self._ctx)
        return out

    def read_walker(self, run: int, walker: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int8)
        _lib.check(_lib.lib().pt2d_read_walker(self._ctx, int(run), int(walker), _p(out)),
                   "pt2d_read_walker", self._ctx)
        return out

    def write(self, what: int, arr) -> None:
        shape, dt = self._spec(what)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, dtype=dt), shape))
        _lib.check(_lib.lib().pt2d_write(self._ctx, what, _p(a), a.nbytes), "pt2d_write",
                   self._ctx)

    def sync(self) -> None:
        _lib.check(_lib.lib().pt2d_sync(self._ctx), "pt2d_sync", self._ctx)

    def kernel_time(self, kind: int) -> tuple[float, int]:
        """(total device ms, launches) of kind 0 = sweep kernel, 1 = swap kernel."""
        ms = C.c_double()
        cnt = C.c_int64()
        _lib.check(_lib.lib().pt2d_kernel_time(self._ctx, int(kind), C.byref(ms), C.byref(cnt)),
                   "pt2d_kernel_time", self._ctx)
        return ms.value, cnt.value

    @property
    def num_colors(self) -> int:
        return int(_lib.lib().pt2d_num_colors(self._ctx))

    @property
    def launch_count(self) -> int:
        return int(_lib.lib().pt2d_launch_count(self._ctx))

    @property
    def tiling(self) -> dict:
        """Sweep tiling chosen at creation: kernel, walkers and threads per CTA,
        walkers per thread."""
        out = (C.c_int32 * 4)()
        _lib.check(_lib.lib().pt2d_tiling(self._ctx, out), "pt2d_tiling", self._ctx)
        return _tiling_dict(out)

    def close(self) -> None:
        if getattr(self, "_ctx", None) and self._ctx.value:
            _lib.lib().pt2d_destroy(self._ctx)
            self._ctx = C.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _tiling_dict(out) -> dict:
    kernel = {1: "global", 2: "smem", 3: "bits", 4: "generic", 5: "generic_smem", 6: "penalty_smem",
              7: "penalty_bits"}[out[0]]
    return dict(kernel=kernel, walkers_per_cta=out[1], threads_per_cta=out[2], walkers_per_thread=out[3])


def plan_tiling(inst: PhysicalInstance, I: int, J: int, runs: int, *, walkers_per_cta: int = 0,
                threads_per_cta: int = 0, walkers_per_thread: int = 0, sweep_kernel: str = "auto") -> dict:
    """The sweep tiling a context would choose (pt2d_plan_tiling), computed on
    the host without a GPU: kernel, walkers and threads per CTA, walkers per
    thread."""
    opt = _lib.Options()
    _lib.lib().pt2d_default_options(C.byref(opt))
    opt.walkers_per_cta = int(walkers_per_cta)
    opt.threads_per_cta = int(threads_per_cta)
    opt.walkers_per_thread = int(walkers_per_thread)
    opt.sweep_kernel = {"auto": 0, "global": 1, "smem": 2, "bits": 3}[sweep_kernel]
    cs = inst.c_struct()
    out = (C.c_int32 * 4)()
    _lib.check(_lib.lib().pt2d_plan_tiling(C.byref(cs), int(I), int(J), int(runs), C.byref(opt), out),
               "pt2d_plan_tiling")
    return _tiling_dict(out)


def _array_spec(what, runs, R, n, T):
    q = runs
    return {
        STATES: ((q, R, n), np.int8), WALKER_AT: ((q, R), np.int32), F: ((q, R), np.int64),
        G: ((q, R), np.int64), COUNTERS: ((4,), np.int64), TRACE_F: ((q, T), np.int64),
        TRACE_G: ((q, T), np.int64), BEST_F: ((q,), np.int64), BEST_EVENT: ((q,), np.int64),
        BEST_STATE: ((q, n), np.int8), SOLVED_EVENT: ((q,), np.int64),
        ACC_P: ((q, R), np.int64), ACC_B: ((q, R), np.int64), SUM_F: ((q, R), np.int64),
        SUM_G: ((q, R), np.int64), N_FEASIBLE: ((q, R), np.int64), COLORS: ((n,), np.int32),
        TARGET: ((q,), np.int64),
    }[what]


class PoolFull(Pt2dError):
    """The batch's device pool has no room for this problem (PT2D_ERR_OOM)."""


class Batch:
    """Batched persistent 2D-PT (pt2d_batch_*): many problems of uneven size in
    one persistent kernel, added and removed between launches."""

    def __init__(self, pool_bytes: int, max_coupling_degree: int = 3, max_runs: int = 4096, *,
                 stream=None, trace_capacity: int = 1024, threads_per_cta: int = 0,
                 spins_in_global: bool = False, sweep_kernel: str = "auto",
                 walkers_per_cta: int = 0, swap_mode: str = "2d", device: int = -1):
        """sweep_kernel: where a run's spins live during an event -- "auto" (int8
        in shared memory, else bit-packed in shared memory, else global memory),
        "global", "smem" (no bit-packed slabs) or "bits" (no int8 shared-memory
        slabs); spins_in_global=True is "global"."""
        L = _lib.lib()
        opt = _lib.Options()
        L.pt2d_default_options(C.byref(opt))
        opt.trace_capacity = int(trace_capacity)
        opt.threads_per_cta = int(threads_per_cta)
        opt.sweep_kernel = 1 if spins_in_global else {"auto": 0, "global": 1, "smem": 2, "bits": 3}[sweep_kernel]
        opt.walkers_per_cta = int(walkers_per_cta)
        opt.swap_mode = SWAP_MODES[swap_mode]
        opt.device = int(device)
        self._stream_obj = stream
        if stream is not None:
            opt.stream = int(getattr(stream, "cuda_stream", stream))
        self.trace_capacity = int(trace_capacity)
        self._b = C.c_void_p()
        _lib.check(L.pt2d_batch_create(C.byref(self._b), int(pool_bytes), int(max_coupling_degree),
                                       int(max_runs), C.byref(opt)), "pt2d_batch_create")
        self._meta = {}
        self._keep = {}

    def instance_bytes(self, inst: PhysicalInstance, I: int, J: int, runs: int) -> int:
        cs = inst.c_struct()
        return int(_lib.lib().pt2d_batch_instance_bytes(self._b, C.byref(cs), int(I), int(J), int(runs)))

    def add(self, inst: PhysicalInstance, beta, P, runs: int, seed: int, target=None) -> int:
        beta = np.ascontiguousarray(beta, dtype=np.float32)
        P = np.ascontiguousarray(P, dtype=np.int32)
        tgt = None if target is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(target, dtype=np.int64), (int(runs),)))
        cs = inst.c_struct()
        bid = C.c_int64()
        st = _lib.lib().pt2d_batch_add(self._b, C.byref(cs), beta.size, _p(beta), P.size, _p(P),
                                       int(runs), int(seed), _p(tgt), C.byref(bid))
        if st == -2:
            raise PoolFull(st, "pt2d_batch_add")
        _lib.check(st, "pt2d_batch_add")
        self._meta[bid.value] = (int(runs), beta.size * P.size, int(inst.n))
        return bid.value

    def remove(self, bid: int) -> None:
        _lib.check(_lib.lib().pt2d_batch_remove(self._b, int(bid)), "pt2d_batch_remove")
        self._meta.pop(bid, None)

    def run(self, events: int, swap_interval: int) -> None:
        st = _lib.lib().pt2d_batch_run(self._b, int(events), int(swap_interval))
        if st != 0:
            raise Pt2dError(st, "pt2d_batch_run", _lib.lib().pt2d_batch_cuda_error(self._b))

    _STORAGE = {"auto": 0, "global": 1, "smem": 2, "bits": 3}

    @staticmethod
    def _shape_dict(sh) -> dict:
        names = {v: k for k, v in Batch._STORAGE.items()}
        return dict(threads_per_cta=sh.threads_per_cta, storage=names[sh.storage],
                    global_width=sh.global_width, balance=sh.balance)

    @property
    def shape(self) -> dict:
        """Launch shape (pt2d_batch_shape): threads_per_cta, storage ("auto",
        "global", "smem", "bits"), global_width, balance."""
        sh = _lib.BatchShape()
        _lib.check(_lib.lib().pt2d_batch_get_shape(self._b, C.byref(sh)), "pt2d_batch_get_shape")
        return self._shape_dict(sh)

    @shape.setter
    def shape(self, value: dict) -> None:
        cur = self.shape
        cur.update(value)
        sh = _lib.BatchShape(int(cur["threads_per_cta"]), self._STORAGE[cur["storage"]],
                             int(cur["global_width"]), int(cur["balance"]))
        _lib.check(_lib.lib().pt2d_batch_set_shape(self._b, C.byref(sh)), "pt2d_batch_set_shape")

    def autotune(self, events: int, swap_interval: int) -> dict:
        """Time candidate launch shapes (each trial advances the chains) and keep
        the fastest; returns it."""
        sh = _lib.BatchShape()
        st = _lib.lib().pt2d_batch_autotune(self._b, int(events), int(swap_interval), C.byref(sh))
        if st != 0:
            raise Pt2dError(st, "pt2d_batch_autotune", _lib.lib().pt2d_batch_cuda_error(self._b))
        return self._shape_dict(sh)

    def read(self, bid: int, what: int) -> np.ndarray:
        runs, R, n = self._meta[bid]
        shape, dt = _array_spec(what, runs, R, n, self.trace_capacity)
        out = np.empty(shape, dtype=dt)
        st = _lib.lib().pt2d_batch_read(self._b, int(bid), what, _p(out), out.nbytes)
        if st != 0:
            raise Pt2dError(st, "pt2d_batch_read", _lib.lib().pt2d_batch_cuda_error(self._b))
        return out

    def sync(self) -> None:
        _lib.check(_lib.lib().pt2d_batch_sync(self._b), "pt2d_batch_sync")

    @property
    def free_bytes(self) -> int:
        return int(_lib.lib().pt2d_batch_free_bytes(self._b))

    @property
    def launch_count(self) -> int:
        return int(_lib.lib().pt2d_batch_launch_count(self._b))

    def close(self) -> None:
        if getattr(self, "_b", None) and self._b.value:
            _lib.lib().pt2d_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (pt2d_server_*)."""

    def __init__(self, pool_bytes: int, max_coupling_degree: int = 3, max_requests: int = 1024,
                 swap_interval: int = 50, events_per_step: int = 10, *, stream=None,
                 threads_per_cta: int = 0, spins_in_global: bool = False,
                 sweep_kernel: str = "auto", swap_mode: str = "2d", device: int = -1):
        """sweep_kernel / spins_in_global: slab storage; swap_mode: as for Batch."""
        L = _lib.lib()
        opt = _lib.Options()
        L.pt2d_default_options(C.byref(opt))
        opt.threads_per_cta = int(threads_per_cta)
        opt.sweep_kernel = 1 if spins_in_global else {"auto": 0, "global": 1, "smem": 2, "bits": 3}[sweep_kernel]
        opt.swap_mode = SWAP_MODES[swap_mode]
        opt.device = int(device)
        self._stream_obj = stream
        if stream is not None:
            opt.stream = int(getattr(stream, "cuda_stream", stream))
        self._s = C.c_void_p()
        _lib.check(L.pt2d_server_create(C.byref(self._s), int(pool_bytes), int(max_coupling_degree),
                                        int(max_requests), int(swap_interval), int(events_per_step),
                                        C.byref(opt)), "pt2d_server_create")

    def submit(self, inst: PhysicalInstance, beta, P, seed: int, target: int, max_sweeps: int) -> int:
        beta = np.ascontiguousarray(beta, dtype=np.float32)
        P = np.ascontiguousarray(P, dtype=np.int32)
        cs = inst.c_struct()
        rid = C.c_int64()
        _lib.check(_lib.lib().pt2d_server_submit(self._s, C.byref(cs), beta.size, _p(beta), P.size,
                                                 _p(P), int(seed), int(target), int(max_sweeps),
                                                 C.byref(rid)), "pt2d_server_submit")
        return rid.value

    def step(self):
        a, q, f = C.c_int32(), C.c_int32(), C.c_int32()
        _lib.check(_lib.lib().pt2d_server_step(self._s, C.byref(a), C.byref(q), C.byref(f)),
                   "pt2d_server_step")
        return a.value, q.value, f.value

    def status(self, rid: int, with_state: bool = False) -> dict:
        st = _lib.RequestStatus()
        L = _lib.lib()
        _lib.check(L.pt2d_server_status(self._s, int(rid), C.byref(st), None), "pt2d_server_status")
        out = {k: getattr(st, k) for k, _ in _lib.RequestStatus._fields_}
        out["state"] = _lib.REQUEST_STATES[st.state]
        if with_state and st.state == 2:
            s = np.zeros(st.n, np.int8)
            _lib.check(L.pt2d_server_status(self._s, int(rid), C.byref(st), _p(s)), "pt2d_server_status")
            out["best_state"] = s
        return out

    def cancel(self, rid: int) -> None:
        _lib.check(_lib.lib().pt2d_server_cancel(self._s, int(rid)), "pt2d_server_cancel")

    def forget(self, rid: int) -> None:
        _lib.check(_lib.lib().pt2d_server_forget(self._s, int(rid)), "pt2d_server_forget")

    @property
    def free_bytes(self) -> int:
        return int(_lib.lib().pt2d_server_free_bytes(self._s))

    def close(self) -> None:
        if getattr(self, "_s", None) and self._s.value:
            _lib.lib().pt2d_server_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adaptive_schedule(inst: PhysicalInstance, *, beta0: float, P0: int, max_rows: int,
                      max_cols: int, sigma_min: float, alpha_beta: float, alpha_P: float,
                      n_chain: int, mcs: int, seed: int, stream=None, device: int = -1):
    """Adaptive beta / P ladders of Algorithm 2 (pt2d_adaptive_schedule).
    Returns (beta float32 [I], P int32 [J], population samples drawn)."""
    prm = _lib.ScheduleParams(float(beta0), int(P0), int(max_rows), int(max_cols), int(n_chain),
                              float(sigma_min), float(alpha_beta), float(alpha_P), int(mcs),
                              int(seed) & ((1 << 64) - 1))
    opt = _lib.Options()
    _lib.lib().pt2d_default_options(C.byref(opt))
    opt.device = int(device)
    if stream is not None:
        opt.stream = int(getattr(stream, "cuda_stream", stream))
    beta = np.zeros(max(int(max_rows), 1), np.float32)
    P = np.zeros(max(int(max_cols), 1), np.int32)
    I, J, k = C.c_int32(), C.c_int32(), C.c_int64()
    cs = inst.c_struct()
    st = _lib.lib().pt2d_adaptive_schedule(
        C.byref(cs), C.byref(prm), C.byref(opt), beta.ctypes.data_as(C.POINTER(C.c_float)),
        C.byref(I), P.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(J), C.byref(k))
    _lib.check(st, "pt2d_adaptive_schedule")
    return beta[:I.value].copy(), P[:J.value].copy(), int(k.value)


def debug_fail_allocations(count: int) -> int:
    """Test hook: make the next `count` workspace / pool allocations fail as
    out of memory (pt2d_debug_fail_allocations); returns the pending count."""
    return int(_lib.lib().pt2d_debug_fail_allocations(int(count)))


def _diag(name, arrays, outs, count):
    st = getattr(_lib.lib(), name)(*[_p(a) for a in arrays], *[_p(o) for o in outs], int(count))
    _lib.check(st, name)


def diag_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    _diag("pt2d_diag_philox", [ctr, key], [out], ctr.shape[0])
    return out


def diag_pt_exp(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    _diag("pt2d_diag_pt_exp", [x], [y], x.size)
    return y


def diag_heatbath(beta, H, r) -> np.ndarray:
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.empty(beta.size, np.int8)
    _diag("pt2d_diag_heatbath", [beta, H, r], [out], beta.size)
    return out


def diag_swap_accept(x, r) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    out = np.empty(x.size, np.int8)
    _diag("pt2d_diag_swap_accept", [x, r], [out], x.size)
    return out


def diag_read_bandwidth(buf, iters: int, out) -> float:
    """Milliseconds for `iters` read passes over a device buffer (any object
    with a CUDA data pointer and byte size, e.g. a torch tensor), L2-cached
    16-byte loads (pt2d_diag_read_bandwidth); `out` is a device buffer of at
    least 4 bytes the probe may write."""
    ms = C.c_float()
    ptr = C.c_void_p(int(buf.data_ptr()))
    nbytes = int(buf.numel() * buf.element_size())
    _lib.check(_lib.lib().pt2d_diag_read_bandwidth(ptr, nbytes, int(iters), C.c_void_p(int(out.data_ptr())),
                                                   C.byref(ms)), "pt2d_diag_read_bandwidth")
    return float(ms.value)
