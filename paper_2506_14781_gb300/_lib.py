"""ctypes binding of libpt2d.so: the C ABI of include/pt2d.h, argument
marshalling only.  Raises if the library has not been built (there is no
fallback implementation)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpt2d.so")

PT2D_OK = 0
ERRORS = {
    -1: "PT2D_ERR_INVALID_ARG",
    -2: "PT2D_ERR_OOM",
    -3: "PT2D_ERR_CUDA",
    -4: "PT2D_ERR_TIMEOUT",
    -5: "PT2D_ERR_STATE",
    -6: "PT2D_ERR_UNSUPPORTED",
}

# readable / writable arrays
STATES, WALKER_AT, F, G, COUNTERS, TRACE_F, TRACE_G, BEST_F, BEST_EVENT, BEST_STATE, \
    SOLVED_EVENT, ACC_P, ACC_B, SUM_F, SUM_G, N_FEASIBLE, COLORS, TARGET = range(1, 19)

SPARSIFY_FIXED, SPARSIFY_MAX_EDGES, SPARSIFY_MAX_DEGREE = 0, 1, 2

EXPORTS = [
    "pt2d_default_options", "pt2d_workspace_size", "pt2d_create", "pt2d_run", "pt2d_read",
    "pt2d_read_walker",
    "pt2d_write", "pt2d_array_bytes", "pt2d_sync", "pt2d_num_colors", "pt2d_tiling", "pt2d_plan_tiling", "pt2d_launch_count",
    "pt2d_destroy", "pt2d_strerror", "pt2d_cuda_error", "pt2d_sparsify", "pt2d_greedy_color",
    "pt2d_diag_philox", "pt2d_diag_pt_exp", "pt2d_diag_heatbath", "pt2d_diag_swap_accept",
    "pt2d_kernel_time", "pt2d_run_noalloc", "pt2d_batch_create", "pt2d_batch_instance_bytes",
    "pt2d_batch_add", "pt2d_batch_remove", "pt2d_batch_run", "pt2d_batch_autotune",
    "pt2d_batch_get_shape", "pt2d_batch_set_shape",
    "pt2d_batch_read", "pt2d_batch_array_bytes", "pt2d_batch_sync", "pt2d_batch_free_bytes",
    "pt2d_batch_launch_count", "pt2d_batch_cuda_error", "pt2d_batch_destroy", "pt2d_batch_poll",
    "pt2d_server_create", "pt2d_server_submit", "pt2d_server_step", "pt2d_server_status",
    "pt2d_server_cancel", "pt2d_server_forget", "pt2d_server_free_bytes", "pt2d_server_destroy",
    "pt2d_adaptive_schedule", "pt2d_onehot_penalty", "pt2d_equality_penalty", "pt2d_diag_read_bandwidth",
    "pt2d_debug_fail_allocations",
]


class Instance(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("cp_ptr", C.c_void_p),
        ("cp_col", C.c_void_p),
        ("cp_J", C.c_void_p),
        ("lk_ptr", C.c_void_p),
        ("lk_col", C.c_void_p),
        ("h", C.c_void_p),
        ("color", C.c_void_p),
        ("lk_w", C.c_void_p),
        ("hk", C.c_void_p),
        ("g0", C.c_int64),
    ]


class Options(C.Structure):
    _fields_ = [
        ("stream", C.c_void_p),
        ("workspace", C.c_void_p),
        ("workspace_bytes", C.c_size_t),
        ("trace_capacity", C.c_int32),
        ("walkers_per_cta", C.c_int32),
        ("threads_per_cta", C.c_int32),
        ("device", C.c_int32),
        ("profile", C.c_int32),
        ("sweep_kernel", C.c_int32),
        ("walkers_per_thread", C.c_int32),
        ("swap_mode", C.c_int32),
    ]


class BatchShape(C.Structure):
    _fields_ = [
        ("threads_per_cta", C.c_int32),
        ("storage", C.c_int32),
        ("global_width", C.c_int32),
        ("balance", C.c_int32),
    ]


class ScheduleParams(C.Structure):
    _fields_ = [
        ("beta0", C.c_double),
        ("P0", C.c_int32),
        ("max_rows", C.c_int32),
        ("max_cols", C.c_int32),
        ("n_chain", C.c_int32),
        ("sigma_min", C.c_double),
        ("alpha_beta", C.c_double),
        ("alpha_P", C.c_double),
        ("mcs", C.c_int32),
        ("seed", C.c_uint64),
    ]


class RequestStatus(C.Structure):
    _fields_ = [
        ("state", C.c_int32),
        ("error", C.c_int32),
        ("n", C.c_int32),
        ("best_f", C.c_int64),
        ("best_event", C.c_int64),
        ("solved_event", C.c_int64),
        ("sweeps_done", C.c_int64),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
    ]


REQUEST_STATES = {0: "queued", 1: "running", 2: "done", 3: "cancelled", 4: "failed"}


class Pt2dError(RuntimeError):
    def __init__(self, status: int, what: str, cuda_error: int = 0):
        self.status = status
        msg = f"{what}: {ERRORS.get(status, status)} ({lib().pt2d_strerror(status).decode()})"
        if cuda_error:
            msg += f" [cudaError {cuda_error}]"
        super().__init__(msg)


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import "
                              f"__graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        L.pt2d_default_options.argtypes = [vp]
        L.pt2d_default_options.restype = None
        L.pt2d_workspace_size.argtypes = [vp, i32, i32, i32, vp, C.POINTER(sz)]
        L.pt2d_create.argtypes = [C.POINTER(vp), vp, i32, vp, i32, vp, i32, vp]
        L.pt2d_run.argtypes = [vp, i64, i32, C.c_uint64]
        L.pt2d_read.argtypes = [vp, i32, vp, sz]
        L.pt2d_write.argtypes = [vp, i32, vp, sz]
        L.pt2d_read_walker.argtypes = [vp, i32, i32, vp]
        L.pt2d_array_bytes.argtypes = [vp, i32]
        L.pt2d_array_bytes.restype = sz
        L.pt2d_sync.argtypes = [vp]
        L.pt2d_num_colors.argtypes = [vp]
        L.pt2d_tiling.argtypes = [vp, C.POINTER(C.c_int32)]
        L.pt2d_plan_tiling.argtypes = [vp, i32, i32, i32, vp, C.POINTER(C.c_int32)]
        L.pt2d_launch_count.argtypes = [vp]
        L.pt2d_launch_count.restype = i64
        L.pt2d_destroy.argtypes = [vp]
        L.pt2d_destroy.restype = None
        L.pt2d_strerror.argtypes = [C.c_int]
        L.pt2d_strerror.restype = C.c_char_p
        L.pt2d_cuda_error.argtypes = [vp]
        L.pt2d_sparsify.argtypes = [i32, vp, i32, i32, C.POINTER(i32), C.POINTER(i64),
                                    C.POINTER(i64), vp, vp, vp, vp, vp, vp]
        L.pt2d_greedy_color.argtypes = [vp, vp, C.POINTER(i32)]
        L.pt2d_diag_philox.argtypes = [vp, vp, vp, i64]
        L.pt2d_diag_pt_exp.argtypes = [vp, vp, i64]
        L.pt2d_diag_heatbath.argtypes = [vp, vp, vp, vp, i64]
        L.pt2d_diag_swap_accept.argtypes = [vp, vp, vp, i64]
        L.pt2d_kernel_time.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(i64)]
        L.pt2d_run_noalloc.argtypes = [vp, i32, vp, i32, vp, i32, i64, i32, C.c_uint64, vp, vp,
                                       vp, vp, vp]
        L.pt2d_batch_create.argtypes = [C.POINTER(vp), sz, i32, i32, vp]
        L.pt2d_batch_instance_bytes.argtypes = [vp, vp, i32, i32, i32]
        L.pt2d_batch_instance_bytes.restype = sz
        L.pt2d_batch_add.argtypes = [vp, vp, i32, vp, i32, vp, i32, C.c_uint64, vp, C.POINTER(i64)]
        L.pt2d_batch_remove.argtypes = [vp, i64]
        L.pt2d_batch_run.argtypes = [vp, i32, i32]
        L.pt2d_batch_autotune.argtypes = [vp, i32, i32, C.POINTER(BatchShape)]
        L.pt2d_debug_fail_allocations.argtypes = [i32]
        L.pt2d_debug_fail_allocations.restype = i32
        L.pt2d_onehot_penalty.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, C.POINTER(i32), vp,
                                          C.POINTER(C.c_int64)]
        L.pt2d_equality_penalty.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, C.POINTER(i32), vp,
                                            C.POINTER(C.c_int64)]
        L.pt2d_diag_read_bandwidth.argtypes = [vp, sz, i32, vp, C.POINTER(C.c_float)]
        L.pt2d_adaptive_schedule.argtypes = [C.POINTER(Instance), C.POINTER(ScheduleParams), vp,
                                             C.POINTER(C.c_float), C.POINTER(i32), C.POINTER(i32),
                                             C.POINTER(i32), C.POINTER(C.c_int64)]
        L.pt2d_batch_get_shape.argtypes = [vp, C.POINTER(BatchShape)]
        L.pt2d_batch_set_shape.argtypes = [vp, C.POINTER(BatchShape)]
        L.pt2d_batch_read.argtypes = [vp, i64, i32, vp, sz]
        L.pt2d_batch_array_bytes.argtypes = [vp, i64, i32]
        L.pt2d_batch_array_bytes.restype = sz
        L.pt2d_batch_sync.argtypes = [vp]
        L.pt2d_batch_free_bytes.argtypes = [vp]
        L.pt2d_batch_free_bytes.restype = sz
        L.pt2d_batch_launch_count.argtypes = [vp]
        L.pt2d_batch_launch_count.restype = i64
        L.pt2d_batch_cuda_error.argtypes = [vp]
        L.pt2d_batch_destroy.argtypes = [vp]
        L.pt2d_batch_destroy.restype = None
        L.pt2d_batch_poll.argtypes = [vp, vp, vp, vp, i32, C.POINTER(i32)]
        L.pt2d_server_create.argtypes = [C.POINTER(vp), sz, i32, i32, i32, i32, vp]
        L.pt2d_server_submit.argtypes = [vp, vp, i32, vp, i32, vp, C.c_uint64, i64, i64,
                                         C.POINTER(i64)]
        L.pt2d_server_step.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.pt2d_server_status.argtypes = [vp, i64, vp, vp]
        L.pt2d_server_cancel.argtypes = [vp, i64]
        L.pt2d_server_forget.argtypes = [vp, i64]
        L.pt2d_server_free_bytes.argtypes = [vp]
        L.pt2d_server_free_bytes.restype = sz
        L.pt2d_server_destroy.argtypes = [vp]
        L.pt2d_server_destroy.restype = None
        for name in EXPORTS:
            getattr(L, name)  # every declared entry point must be exported
        _lib = L
    return _lib


def check(status: int, what: str, ctx=None) -> None:
    if status != PT2D_OK:
        cuda_err = lib().pt2d_cuda_error(ctx) if ctx else 0
        raise Pt2dError(status, what, cuda_err)
