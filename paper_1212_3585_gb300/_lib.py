"""ctypes binding of libaderweno.so (include/aderweno.h).  Argument marshalling only: every
step of the solver runs in the library's CUDA kernels.  Importing this module does not need a
GPU; loading the library does need it to have been built (``paper_1212_3585_gb300.build``)."""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libaderweno.so")

AW_OK, AW_EINVAL, AW_ENOMEM, AW_ECUDA, AW_ENONPHYSICAL, AW_ETIMEOUT, AW_ESTATE = 0, -1, -2, -3, -4, -5, -6
AW_ELIMIT = -7
AW_TUNE_PREDICTOR, AW_TUNE_FLUX, AW_TUNE_TRIALS = 0, 1, 2
AW_PDE_EULER, AW_PDE_MHD_GLM, AW_PDE_LINADV = 0, 1, 2
AW_BC_PERIODIC, AW_BC_TRANSMISSIVE, AW_BC_REFLECTIVE, AW_BC_INFLOW = 0, 1, 2, 3
AW_FLUX_RUSANOV, AW_FLUX_OSHER = 0, 1
AW_IC_CONST, AW_IC_VORTEX, AW_IC_EXPLOSION, AW_IC_OT, AW_IC_RP4, AW_IC_FOURIER = 0, 1, 2, 3, 4, 5
AW_INTERNAL_WENO, AW_INTERNAL_PREDICTOR, AW_INTERNAL_CHI, AW_INTERNAL_FLUX = 0, 1, 2, 3
AW_BATCH_MAX = 8


class AwConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("pde", C.c_int32), ("M", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("gamma", C.c_double), ("c_h", C.c_double),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", C.c_int32 * 6),
        ("refine_factor", C.c_int32), ("lmax", C.c_int32),
        ("chi_ref", C.c_double), ("chi_rec", C.c_double), ("eps_ind", C.c_double), ("cfl", C.c_double),
        ("picard_iters", C.c_int32), ("flux", C.c_int32), ("auto_regrid", C.c_int32), ("reserved", C.c_int32),
        ("adv", C.c_double * 3),
        ("inflow", C.c_double * 9),
    ]


class AwStats(C.Structure):
    _fields_ = [
        ("level0_steps", C.c_int64), ("cell_updates", C.c_int64), ("updates_per_level", C.c_int64 * 8),
        ("last_dt0", C.c_double), ("t", C.c_double),
    ]


class AwSrvInfo(C.Structure):
    _fields_ = [("cell_updates", C.c_int64), ("level0_steps", C.c_int64), ("footprint_bytes", C.c_int64),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("total_ms", C.c_double),
                ("requeues", C.c_int64), ("peak_bytes", C.c_int64), ("grows", C.c_int64)]


class AwSrvSummary(C.Structure):
    _fields_ = [("done", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("solves_per_s", C.c_double),
                ("cell_updates_per_s", C.c_double), ("requeues", C.c_int64), ("budget_bytes", C.c_int64),
                ("peak_reserved_bytes", C.c_int64), ("grows", C.c_int64)]


class AwLaunchParams(C.Structure):
    _fields_ = [("pass_min_cells", C.c_int64), ("tile8_min_cells", C.c_int64), ("small_ctas_per_sm", C.c_int32),
                ("fuse_flux_update", C.c_int32), ("autotune", C.c_int32), ("persistent", C.c_int32),
                ("graph_steps", C.c_int32), ("reserved", C.c_int32)]


class AwTuneEntry(C.Structure):
    _fields_ = [("dim", C.c_int32), ("M", C.c_int32), ("pde", C.c_int32), ("flux", C.c_int32), ("kernel", C.c_int32),
                ("size_class", C.c_int32), ("choice", C.c_int32), ("trials", C.c_int32 * 2), ("inherited", C.c_int32),
                ("ns_per_cell", C.c_double * 2)]


class AwCell(C.Structure):
    _fields_ = [("level", C.c_int32), ("status", C.c_int32), ("i", C.c_int32), ("j", C.c_int32), ("k", C.c_int32)]


# name -> (restype, argtypes); every symbol declared in include/aderweno.h
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i8p = C.POINTER(C.c_int8)
SIGNATURES = {
    "aw_create": (C.c_int, [C.POINTER(AwConfig), C.c_size_t, C.POINTER(_vp)]),
    "aw_destroy": (None, [_vp]),
    "aw_last_error": (C.c_char_p, []),
    "aw_set_initial": (C.c_int, [_vp, C.c_int32, _dp, C.c_int32, C.c_int32]),
    "aw_set_cell_averages": (C.c_int, [_vp, _dp, C.c_int64]),
    "aw_step": (C.c_int, [_vp, C.c_double, C.POINTER(AwStats)]),
    "aw_step_dt": (C.c_int, [_vp, C.c_double, C.POINTER(AwStats)]),
    "aw_advance_to": (C.c_int, [_vp, C.c_double, C.POINTER(AwStats)]),
    "aw_advance_graph": (C.c_int, [_vp, C.c_double, C.c_int32, C.POINTER(AwStats)]),
    "aw_get_launch_params": (C.c_int, [C.POINTER(AwLaunchParams)]),
    "aw_set_launch_params": (C.c_int, [C.POINTER(AwLaunchParams)]),
    "aw_get_tuning": (C.c_int, [C.POINTER(AwTuneEntry), C.c_int32, C.POINTER(C.c_int32)]),
    "aw_reset_tuning": (C.c_int, []),
    "aw_compute_dt": (C.c_int, [_vp, _dp]),
    "aw_regrid": (C.c_int, [_vp, C.c_int32]),
    "aw_regrid_with_flags": (C.c_int, [_vp, _i8p, C.c_int64, C.c_int32]),
    "aw_compute_flags": (C.c_int, [_vp, C.c_int32, _i8p, C.c_int64, _i64p]),
    "aw_get_counts": (C.c_int, [_vp, _i64p, _i64p, _i64p, _i64p]),
    "aw_read_cells": (C.c_int, [_vp, C.POINTER(AwCell), _dp, C.c_int64, _i64p]),
    "aw_read_internal": (C.c_int, [_vp, C.c_int32, C.c_int32, _dp, C.c_int64, _i64p]),
    "aw_get_time": (C.c_int, [_vp, _dp]),
    "aw_totals": (C.c_int, [_vp, _dp]),
    "aw_num_vars": (C.c_int, [_vp]),
    "aw_sync": (C.c_int, [_vp]),
    "aw_reset": (C.c_int, [_vp]),
    "aw_set_memory_limit": (C.c_int, [_vp, C.c_int64]),
    "aw_get_memory": (C.c_int, [_vp, _i64p, _i64p, _i64p]),
    "aw_graph_stats": (C.c_int, [_vp, _i64p, _i64p, _i64p]),
    "aw_set_profiling": (C.c_int, [_vp, C.c_int32]),
    "aw_kernel_times": (C.c_int, [_vp, _dp, _i64p]),
    "aw_srv_create": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(_vp)]),
    "aw_srv_set_batching": (C.c_int, [_vp, C.c_int32]),
    "aw_srv_submit": (C.c_int, [_vp, C.POINTER(AwConfig), C.c_int32, _dp, C.c_int32, C.c_double, _i64p]),
    "aw_srv_poll": (C.c_int, [_vp, C.c_int64, C.POINTER(C.c_int32)]),
    "aw_srv_wait_all": (C.c_int, [_vp]),
    "aw_srv_result": (C.c_int, [_vp, C.c_int64, C.POINTER(AwCell), _dp, C.c_int64, _i64p, C.POINTER(AwSrvInfo)]),
    "aw_srv_stats": (C.c_int, [_vp, C.POINTER(AwSrvSummary)]),
    "aw_srv_last_error": (C.c_char_p, []),
    "aw_srv_destroy": (None, [_vp]),
    "aw_selftest_reciprocal": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t]),
    "aw_selftest_flux_math": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t]),
    "aw_cfl_dt_noalloc": (C.c_int, [C.POINTER(AwConfig), C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t]),
    "aw_tables_host": (C.c_int, [C.c_int32, C.c_int32, _dp, C.c_int64, C.POINTER(C.c_int64)]),
    "aw_kernel_launches": (C.c_int64, [_vp]),
    "aw_advance_batch": (C.c_int, [C.POINTER(_vp), C.c_int32, C.c_double, C.c_size_t, C.POINTER(AwStats),
                                   C.POINTER(C.c_int32)]),
    "aw_step_batch": (C.c_int, [C.POINTER(_vp), C.c_int32, _dp, C.c_size_t, C.POINTER(AwStats),
                                C.POINTER(C.c_int32)]),
}

_lib = None


class AwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"aderweno error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libaderweno.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1212_3585_gb300.build` "
                           "(the solver has no CPU fallback)")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(rc):
    if rc != AW_OK:
        raise AwError(rc, _lib.aw_last_error().decode())
    return rc
