"""ctypes declarations of libpatbp.so (include/pat_bp.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1501_03869_gb300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpatbp.so")

PAT_OK, PAT_ERR_INVALID, PAT_ERR_OOM, PAT_ERR_CUDA = 0, 1, 2, 3
PAT_ERR_TIMEOUT, PAT_ERR_BUSY, PAT_ERR_NOT_FOUND, PAT_PENDING = 4, 5, 6, 7
PAT_F32, PAT_BF16, PAT_F16 = 0, 1, 2
PAT_FLAG_COMPACT_OUT = 0x1
PAT_FLAG_TILE_128 = 0x10
PAT_FLAG_TILE_256 = 0x20

# Every symbol include/pat_bp.h declares (checked by the CPU test suite).
EXPORTS = (
    "pat_status_str", "pat_last_error", "pat_bp_create", "pat_bp_reconstruct",
    "pat_bp_preprocess", "pat_bp_gather",
    "pat_bp_reconstruct_host", "pat_bp_reserve", "pat_bp_sync", "pat_bp_info",
    "pat_bp_table", "pat_bp_destroy", "pat_fmm_host", "pat_fmm_gpu", "pat_table_host", "pat_bp_set_solid_angle",
    "pat_test_wait_timeout", "pat_test_gather_only", "pat_plan_create", "pat_plan_execute", "pat_plan_sync",
    "pat_plan_info", "pat_plan_destroy", "pat_bp_reconstruct_multi", "pat_bp_autotune",
    "pat_bp_evict", "pat_bp_restore", "pat_srv_create", "pat_srv_register", "pat_srv_submit",
    "pat_srv_poll", "pat_srv_stats", "pat_srv_destroy", "pat_bp_reconstruct_noalloc",
    "pat_bp_create_constant", "pat_srv_set_budget", "pat_probe_l2_to_smem",
)
PAT_FLAG_HOST_MIRROR = 0x100
PAT_FLAG_STAGED_SINGLE = 0x200
PAT_FLAG_NO_WINDOW = 0x1000
PAT_FLAG_FMM_SECOND_ORDER = 0x400
PAT_FLAG_GPU_TABLE = 0x800
PAT_PLAN_AUTOTUNE = 0x1
PAT_PLAN_GRAPH = 0x2


class PatGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double),
                ("origin", ctypes.c_double * 3)]


class PatInfo(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int64), ("grid_total", ctypes.c_int64),
                ("n_sensors", ctypes.c_int), ("n_samples", ctypes.c_int),
                ("n_samples_pad", ctypes.c_int), ("tile_pix", ctypes.c_int),
                ("n_tiles", ctypes.c_int), ("window", ctypes.c_int), ("split", ctypes.c_int),
                ("sensor_warps", ctypes.c_int), ("table_bytes", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("delays", ctypes.c_int),
                ("c0", ctypes.c_double), ("solid_angle", ctypes.c_int), ("gpu_table", ctypes.c_int)]


class PatPlanInfo(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int), ("frames_per_unit", ctypes.c_int),
                ("sensors_per_stage", ctypes.c_int), ("stages", ctypes.c_int),
                ("smem_budget_kb", ctypes.c_int), ("grid", ctypes.c_int),
                ("n_units", ctypes.c_int64), ("tuned", ctypes.c_int), ("graph", ctypes.c_int),
                ("tune_ms", ctypes.c_double), ("n_classes", ctypes.c_int), ("fb_mask", ctypes.c_int)]


class PatSrvCfg(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("max_batch_frames", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("stall_us", ctypes.c_int)]


class PatSrvStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("uploads", ctypes.c_uint64), ("evictions", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_batch_frames", ctypes.c_double), ("resident_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t)]


class PatError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        super().__init__(f"{what}: status {status} ({detail})")


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_u = ctypes.c_uint
_d = ctypes.c_double
_u64 = ctypes.c_uint64


def load():
    """Load libpatbp.so once; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        lib.pat_status_str.restype = ctypes.c_char_p
        lib.pat_status_str.argtypes = [_i]
        lib.pat_last_error.restype = ctypes.c_char_p
        lib.pat_last_error.argtypes = []
        lib.pat_bp_create.restype = _i
        lib.pat_bp_create.argtypes = [_vp, ctypes.POINTER(PatGrid), _vp, _i, _vp, _vp, _d, _i, _u,
                                      ctypes.POINTER(_vp)]
        lib.pat_bp_create_constant.restype = _i
        lib.pat_bp_create_constant.argtypes = [_d, ctypes.POINTER(PatGrid), _vp, _i, _vp, _vp, _d,
                                               _i, _u, ctypes.POINTER(_vp)]
        lib.pat_bp_reconstruct.restype = _i
        lib.pat_bp_reconstruct.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp]
        lib.pat_bp_preprocess.restype = _i
        lib.pat_bp_preprocess.argtypes = [_vp, _vp, _i, _vp, _i, _vp]
        lib.pat_bp_gather.restype = _i
        lib.pat_bp_gather.argtypes = [_vp, _i, _vp, _vp]
        lib.pat_bp_reconstruct_host.restype = _i
        lib.pat_bp_reconstruct_host.argtypes = [_vp, _vp, _i, _vp, _i, _vp]
        lib.pat_bp_reserve.restype = _i
        lib.pat_bp_reserve.argtypes = [_vp, _i, _i]
        lib.pat_bp_sync.restype = _i
        lib.pat_bp_sync.argtypes = [_vp, _vp]
        lib.pat_bp_info.restype = _i
        lib.pat_bp_info.argtypes = [_vp, ctypes.POINTER(PatInfo)]
        lib.pat_bp_table.restype = _i
        lib.pat_bp_table.argtypes = [_vp, _vp, _vp, _vp]
        lib.pat_bp_destroy.restype = _i
        lib.pat_bp_destroy.argtypes = [_vp]
        lib.pat_fmm_host.restype = _i
        lib.pat_fmm_host.argtypes = [_vp, ctypes.POINTER(PatGrid), _vp, _i, _vp]
        lib.pat_fmm_gpu.restype = _i
        lib.pat_fmm_gpu.argtypes = [_vp, ctypes.POINTER(PatGrid), _vp, _i, _vp]
        lib.pat_bp_set_solid_angle.restype = _i
        lib.pat_bp_set_solid_angle.argtypes = [_vp, _vp, _vp, ctypes.c_double]
        lib.pat_table_host.restype = _i
        lib.pat_table_host.argtypes = [_vp, ctypes.POINTER(PatGrid), _vp, _i, _vp, _d, _i, _u,
                                       ctypes.POINTER(PatInfo), _vp, _vp, _vp]
        _pp = ctypes.POINTER(_vp)
        lib.pat_plan_create.restype = _i
        lib.pat_plan_create.argtypes = [_pp, ctypes.POINTER(_i), _i, _i, _u, _pp]
        lib.pat_plan_execute.restype = _i
        lib.pat_plan_execute.argtypes = [_vp, _pp, _pp, _pp, _vp]
        lib.pat_plan_sync.restype = _i
        lib.pat_plan_sync.argtypes = [_vp, _vp]
        lib.pat_plan_info.restype = _i
        lib.pat_plan_info.argtypes = [_vp, ctypes.POINTER(PatPlanInfo)]
        lib.pat_plan_destroy.restype = _i
        lib.pat_plan_destroy.argtypes = [_vp]
        lib.pat_bp_reconstruct_multi.restype = _i
        lib.pat_bp_reconstruct_multi.argtypes = [_pp, _pp, _i, _pp, ctypes.POINTER(_i), _pp, _i, _vp]
        lib.pat_bp_autotune.restype = _i
        lib.pat_bp_autotune.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp]
        lib.pat_bp_reconstruct_noalloc.restype = _i
        lib.pat_bp_reconstruct_noalloc.argtypes = [_vp, _vp, _i, _vp, _i, _vp, _vp]
        lib.pat_bp_evict.restype = _i
        lib.pat_bp_evict.argtypes = [_vp]
        lib.pat_bp_restore.restype = _i
        lib.pat_bp_restore.argtypes = [_vp, _vp]
        lib.pat_srv_create.restype = _i
        lib.pat_srv_create.argtypes = [ctypes.c_size_t, ctypes.POINTER(PatSrvCfg), _pp]
        lib.pat_srv_register.restype = _i
        lib.pat_srv_register.argtypes = [_vp, _vp, ctypes.POINTER(PatGrid), _vp, _i, _vp, _vp, _d, _i,
                                         _u, ctypes.POINTER(_i)]
        lib.pat_srv_submit.restype = _i
        lib.pat_srv_submit.argtypes = [_vp, _i, _vp, _i, _vp, _vp, ctypes.POINTER(_u64)]
        lib.pat_srv_poll.restype = _i
        lib.pat_srv_poll.argtypes = [_vp, _u64, _i, ctypes.POINTER(_d)]
        lib.pat_srv_stats.restype = _i
        lib.pat_srv_stats.argtypes = [_vp, ctypes.POINTER(PatSrvStats)]
        lib.pat_srv_destroy.restype = _i
        lib.pat_srv_destroy.argtypes = [_vp]
        lib.pat_srv_set_budget.restype = _i
        lib.pat_srv_set_budget.argtypes = [_vp, ctypes.c_size_t]
        lib.pat_probe_l2_to_smem.restype = _i
        lib.pat_probe_l2_to_smem.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.pat_test_wait_timeout.restype = _i
        lib.pat_test_wait_timeout.argtypes = [_u64]
        lib.pat_test_gather_only.restype = _i
        lib.pat_test_gather_only.argtypes = [_vp, _vp]
        _lib = lib
        return lib


def check(status, what):
    if status != PAT_OK:
        lib = load()
        detail = lib.pat_last_error().decode(errors="replace")
        raise PatError(status, what, f"{lib.pat_status_str(status).decode()}: {detail}")


def make_grid(shape, dx, origin):
    """pat_grid of a numpy-shaped ([nz,] ny, nx) grid."""
    g = PatGrid()
    g.ndim = len(shape)
    n = list(shape[::-1]) + [1] * (3 - len(shape))
    for d in range(3):
        g.n[d] = int(n[d])
        g.origin[d] = float(origin[d]) if d < len(origin) else 0.0
    g.dx = float(dx)
    return g
