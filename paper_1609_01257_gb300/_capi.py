"""ctypes view of the C ABI declared in ``include/rng.h``.

Argument marshalling only: every step of the generator runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import builder as _build

c_u64 = ctypes.c_uint64
c_u32 = ctypes.c_uint32
c_i32 = ctypes.c_int32
c_int = ctypes.c_int
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p
c_cp = ctypes.c_char_p
P_u64 = ctypes.POINTER(ctypes.c_uint64)

RNG_OK, RNG_EINVAL, RNG_ENOMEM, RNG_ECUDA, RNG_ESTATE, RNG_ETIMEOUT, RNG_EBUDGET, RNG_ESINK = range(8)
RNG_PROF_SORT_NAME, RNG_PROF_SORT_TIME, RNG_PROF_SORT_DESC = 0, 1, 0x10
RNG_HOST_HUGE_PAGES = 1


class RngErr(ctypes.Structure):
    _fields_ = [("code", c_int), ("msg", ctypes.c_char * 256)]


class RngOpts(ctypes.Structure):
    _fields_ = [
        ("struct_size", c_u32),
        ("values_per_thread", c_u32),
        ("block_threads", c_u32),
        ("fuse_init", c_u32),
        ("stream_offset", c_u64),
        ("device_buffer_bytes", c_u64),
        ("host_slots", c_u32),
        ("profiling", c_u32),
        ("compute_stream", c_vp),
        ("device", c_i32),
        ("store_policy", c_u32),
        ("host_wait_ms", c_u32),
        ("store_width", c_u32),
        ("grid_blocks", c_u32),
        ("host_path", c_u32),
        ("host_consumers", c_u32),
        ("output_mode", c_u32),
    ]


class RngHostStats(ctypes.Structure):
    _fields_ = [
        ("chunks", c_u64),
        ("consumers", c_u32),
        ("slots", c_u32),
        ("wall_s", ctypes.c_double),
        ("producer_wait_s", ctypes.c_double),
        ("copy_wait_s", ctypes.c_double),
        ("consume_s", ctypes.c_double),
    ]


class RngLaunchInfo(ctypes.Structure):
    _fields_ = [("struct_size", c_u32), ("kernel", c_u32), ("values_per_thread", c_u32),
                ("block_threads", c_u32), ("grid_blocks", c_u32), ("row_buffers", c_u32), ("band_rows", c_u64)]


KERNEL_NAMES = {0: "register", 1: "staged", 2: "bulk"}


class RngBatchOpts(ctypes.Structure):
    _fields_ = [
        ("struct_size", c_u32),
        ("values_per_thread", c_u32),
        ("block_threads", c_u32),
        ("tune_reps", c_u32),
        ("stream", c_vp),
        ("device", c_i32),
        ("mode", c_u32),
        ("stores", c_u32),
    ]


class RngServerOpts(ctypes.Structure):
    _fields_ = [
        ("struct_size", c_u32),
        ("max_active", c_u32),
        ("hbm_budget_bytes", c_u64),
        ("step_bytes", c_u64),
        ("max_steps_in_flight", c_u32),
        ("values_per_thread", c_u32),
        ("max_units_per_step", c_u32),
        ("device", c_i32),
        ("stream", c_vp),
        ("mode", c_u32),
    ]


class RngServerStats(ctypes.Structure):
    _fields_ = [(n, c_u64) for n in (
        "submitted", "completed", "rejected", "released", "steps", "bytes_generated",
        "pending", "active", "bytes_in_use", "peak_bytes_in_use", "peak_active")]


P_err = ctypes.POINTER(ctypes.POINTER(RngErr))

SINK_FN = ctypes.CFUNCTYPE(c_int, c_vp, c_u64, c_u64, c_u64, c_u64, c_u64, P_u64)

# name -> (argtypes, restype); the complete exported surface of include/rng.h.
SIGNATURES = {
    "rng_err_clear": ([P_err], None),
    "rng_strerror": ([c_int], c_cp),
    "rng_live_objects": ([], ctypes.c_long),
    "rng_launch_count": ([], c_u64),
    "rng_opts_default": ([ctypes.POINTER(RngOpts)], None),
    "rng_create": ([c_u64, c_u64, ctypes.POINTER(RngOpts), ctypes.POINTER(c_vp), P_err], c_int),
    "rng_init": ([c_vp, P_err], c_int),
    "rng_generate": ([c_vp, c_u64, c_vp, c_vp, P_err], c_int),
    "rng_generate_sink": ([c_vp, c_u64, SINK_FN, c_vp, P_err], c_int),
    "rng_generate_ring": ([c_vp, c_u64, c_vp, c_u64, P_err], c_int),
    "rng_generate_fd": ([c_vp, c_u64, c_int, P_err], c_int),
    "rng_generate_host_checksum": ([c_vp, c_u64, c_vp, c_vp, P_err], c_int),
    "rng_host_stats_get": ([c_vp, c_vp], c_int),
    "rng_generate_checksum": ([c_vp, c_u64, c_vp, c_vp, P_err], c_int),
    "rng_skip": ([c_vp, c_u64, P_err], c_int),
    "rng_position": ([c_vp, P_u64], c_int),
    "rng_streams": ([c_vp, P_u64], c_int),
    "rng_get_state": ([c_vp, c_vp, P_err], c_int),
    "rng_set_state": ([c_vp, c_vp, c_u64, P_err], c_int),
    "rng_sync": ([c_vp, P_err], c_int),
    "rng_compute_stream": ([c_vp], c_vp),
    "rng_launch_config": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32), ctypes.POINTER(c_u32)], c_int),
    "rng_last_launch": ([c_vp, ctypes.POINTER(RngLaunchInfo), P_err], c_int),
    "rng_destroy": ([c_vp], None),
    "rng_prof_new": ([], c_vp),
    "rng_prof_add": ([c_vp, c_cp, c_cp, c_dbl, c_dbl], c_int),
    "rng_prof_set_elapsed": ([c_vp, c_dbl], c_int),
    "rng_prof_calc": ([c_vp, P_err], c_int),
    "rng_prof_num_aggregates": ([c_vp], ctypes.c_size_t),
    "rng_prof_aggregate": ([c_vp, ctypes.c_size_t, ctypes.POINTER(c_cp), ctypes.POINTER(c_dbl),
                            ctypes.POINTER(c_dbl)], c_int),
    "rng_prof_num_overlaps": ([c_vp], ctypes.c_size_t),
    "rng_prof_overlap": ([c_vp, ctypes.c_size_t, ctypes.POINTER(c_cp), ctypes.POINTER(c_cp),
                          ctypes.POINTER(c_dbl)], c_int),
    "rng_prof_total": ([c_vp], c_dbl),
    "rng_prof_effective": ([c_vp], c_dbl),
    "rng_prof_elapsed": ([c_vp], c_dbl),
    "rng_prof_summary": ([c_vp, c_int, c_int], c_cp),
    "rng_prof_export": ([c_vp, c_cp, P_err], c_int),
    "rng_prof_destroy": ([c_vp], None),
    "rng_profiler": ([c_vp, P_err], c_vp),
    "rng_profile_summary": ([c_vp, c_int, c_int, P_err], c_cp),
    "rng_profile_export": ([c_vp, c_cp, P_err], c_int),
    "rng_profile_reset": ([c_vp, P_err], c_int),
    "rng_profile_stat": ([c_vp, c_cp, P_u64, ctypes.POINTER(c_dbl), P_err], c_int),
    "rng_batch_opts_default": ([ctypes.POINTER(RngBatchOpts)], None),
    "rng_batch_create": ([c_u32, P_u64, P_u64, P_u64, ctypes.POINTER(c_vp), ctypes.POINTER(RngBatchOpts),
                          ctypes.POINTER(c_vp), P_err], c_int),
    "rng_batch_run": ([c_vp, P_err], c_int),
    "rng_batch_sync": ([c_vp, P_err], c_int),
    "rng_batch_stores": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32)], c_int),
    "rng_batch_config": ([c_vp, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32), ctypes.POINTER(c_u32),
                          P_u64, ctypes.POINTER(c_u32), ctypes.POINTER(c_dbl)], c_int),
    "rng_batch_stream": ([c_vp], c_vp),
    "rng_batch_destroy": ([c_vp], None),
    "rng_batch_generate_noalloc": ([c_u32, P_u64, P_u64, P_u64, ctypes.POINTER(c_vp), c_vp, P_err], c_int),
    "rng_server_opts_default": ([ctypes.POINTER(RngServerOpts)], None),
    "rng_server_create": ([ctypes.POINTER(RngServerOpts), ctypes.POINTER(c_vp), P_err], c_int),
    "rng_server_submit": ([c_vp, c_u64, c_u64, c_u64, P_u64, P_err], c_int),
    "rng_server_submit_ex": ([c_vp, c_u64, c_u64, c_u64, c_u32, c_u64, P_u64, P_err], c_int),
    "rng_server_poll": ([c_vp, c_u32, P_u64, ctypes.POINTER(c_vp), ctypes.POINTER(c_dbl),
                         ctypes.POINTER(c_u32), c_u32, P_err], c_int),
    "rng_server_read": ([c_vp, c_u64, c_u64, c_u64, c_vp, P_err], c_int),
    "rng_server_release": ([c_vp, c_u64, P_err], c_int),
    "rng_server_get_stats": ([c_vp, ctypes.POINTER(RngServerStats)], c_int),
    "rng_server_destroy": ([c_vp], None),
    "rng_host_alloc": ([ctypes.c_size_t, c_u32, ctypes.POINTER(c_vp), P_err], c_int),
    "rng_host_free": ([c_vp], c_int),
}


class RngError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code
        self.msg = msg


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Loads the built library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: run `python -m paper_1609_01257_gb300.builder` "
                "(or __graft_entry__.build()) first; there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def check(fn, *args):
    """Calls a status-returning entry point with an error slot; raises RngError."""
    err = ctypes.POINTER(RngErr)()
    rc = fn(*args, ctypes.byref(err))
    if rc != RNG_OK:
        msg = err.contents.msg.decode(errors="replace") if err else load().rng_strerror(rc).decode()
        load().rng_err_clear(ctypes.byref(err))
        raise RngError(rc, msg)
    if err:
        load().rng_err_clear(ctypes.byref(err))
    return rc
