"""ctypes declarations of the libnf C ABI (include/nf.h).

Loading fails loudly when the shared library has not been built: there is no
fallback implementation of any step in Python.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnf.so")

NF_OK, NF_EINVAL, NF_ERANGE, NF_ENOMEM, NF_ECUDA, NF_ESTATE, NF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
NF_SOFT_PLUMMER, NF_SOFT_SPLINE = 0, 1
SOFTENINGS = {"plummer": NF_SOFT_PLUMMER, "spline": NF_SOFT_SPLINE}
NF_PREC_FP32, NF_PREC_FP32_COMP, NF_PREC_FP64_REF, NF_PREC_FP32_COMP_PAIR = 0, 1, 2, 3
PRECISIONS = {"fp32": NF_PREC_FP32, "fp32_comp": NF_PREC_FP32_COMP, "fp64": NF_PREC_FP64_REF,
              "fp32_comp_pair": NF_PREC_FP32_COMP_PAIR}

# every entry point include/nf.h declares
EXPORTS = ("nf_init", "nf_bin_particles", "nf_compute_accel", "nf_compute_accel_f64",
           "nf_compute_accel_vjp", "nf_accel_host", "nf_get_stats", "nf_set_tuning",
           "nf_get_tuning", "nf_autotune", "nf_copy_binning", "nf_bin_cells_noalloc",
           "nf_compute_accel_density", "nf_set_box_masses", "nf_kick", "nf_drift", "nf_timestep",
           "nf_kdk_step", "nf_far_init", "nf_compute_far", "nf_init_slab", "nf_slab_export",
           "nf_slab_import", "nf_slab_of",
           "nf_last_error", "nf_status_string", "nf_free")


class nf_stats(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("interactions", ctypes.c_int64), ("max_occupancy", ctypes.c_int64),
                ("n_items", ctypes.c_int64), ("momentum", ctypes.c_double * 3),
                ("abs_momentum", ctypes.c_double), ("bin_ms", ctypes.c_double),
                ("pair_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("far_ms", ctypes.c_double), ("far_conv_ms", ctypes.c_double),
                ("n_pencils", ctypes.c_int64), ("n_small", ctypes.c_int64)]


class nf_tuning(ctypes.Structure):
    _fields_ = [("sinks_per_lane", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("vjp_sinks_per_lane", ctypes.c_int), ("source_tile", ctypes.c_int),
                ("use_pencils", ctypes.c_int), ("small_items", ctypes.c_int)]


class NFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def _status_name(code: int) -> str:
    names = {0: "NF_OK", -1: "NF_EINVAL", -2: "NF_ERANGE", -3: "NF_ENOMEM", -4: "NF_ECUDA",
             -5: "NF_ESTATE", -6: "NF_ETIMEOUT"}
    return names.get(code, f"NF_{code}")


def load(path: str | None = None):
    """Load libnf.so (built by ``paper_2110_11398_gb300.build``) and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libnf.so is not built ({p} missing); run "
                "`python -m paper_2110_11398_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(p)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        lib.nf_init.argtypes = [P(vp), i32, i32, P(dbl), P(i32), i32, P(dbl), i32, i32, i64]
        lib.nf_bin_particles.argtypes = [vp, vp, vp, dbl, i64, P(i64), vp]
        lib.nf_compute_accel.argtypes = [vp, vp, vp]
        lib.nf_compute_accel_f64.argtypes = [vp, vp, vp]
        lib.nf_compute_accel_vjp.argtypes = [vp, vp, vp, vp]
        lib.nf_compute_accel_density.argtypes = [vp, vp, vp, P(dbl), vp]
        lib.nf_set_box_masses.argtypes = [vp, P(dbl)]
        lib.nf_kick.argtypes = [vp, vp, vp, dbl, vp]
        lib.nf_drift.argtypes = [vp, vp, vp, dbl, vp]
        lib.nf_timestep.argtypes = [vp, vp, vp, dbl, P(dbl), vp]
        lib.nf_kdk_step.argtypes = [vp, vp, vp, vp, vp, dbl, dbl, P(i64), vp]
        lib.nf_far_init.argtypes = [vp, i32, vp]
        lib.nf_compute_far.argtypes = [vp, vp, i32, vp]
        lib.nf_accel_host.argtypes = [vp, vp, vp, dbl, i64, P(i64), vp, vp]
        lib.nf_get_stats.argtypes = [vp, P(nf_stats)]
        lib.nf_set_tuning.argtypes = [vp, P(nf_tuning)]
        lib.nf_get_tuning.argtypes = [vp, P(nf_tuning)]
        lib.nf_autotune.argtypes = [vp, i32, P(nf_tuning), vp]
        lib.nf_copy_binning.argtypes = [vp, vp, vp, vp, vp]
        lib.nf_bin_cells_noalloc.argtypes = [vp, vp, dbl, i64, dbl, i32, vp, vp, vp, vp]
        lib.nf_init_slab.argtypes = [P(vp), i32, dbl, i32, i32, dbl, i32, i32, i64, i32, i32]
        lib.nf_slab_export.argtypes = [vp, i32, vp, vp, i64, P(i64), vp]
        lib.nf_slab_import.argtypes = [vp, vp, vp, i64, vp, vp, i64, vp]
        lib.nf_slab_of.argtypes = [vp, i64, dbl, i32, vp, vp]
        lib.nf_last_error.argtypes = [vp]
        lib.nf_last_error.restype = ctypes.c_char_p
        lib.nf_status_string.argtypes = [i32]
        lib.nf_status_string.restype = ctypes.c_char_p
        lib.nf_free.argtypes = [vp]
        lib.nf_free.restype = None
        for name in ("nf_init", "nf_bin_particles", "nf_compute_accel", "nf_compute_accel_f64",
                     "nf_compute_accel_vjp", "nf_accel_host", "nf_get_stats", "nf_set_tuning",
                     "nf_get_tuning", "nf_autotune", "nf_copy_binning", "nf_bin_cells_noalloc",
                     "nf_far_init", "nf_compute_far", "nf_compute_accel_density", "nf_set_box_masses", "nf_kick", "nf_drift",
                     "nf_timestep", "nf_kdk_step", "nf_init_slab", "nf_slab_export", "nf_slab_import",
                     "nf_slab_of"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def check(rc: int, ctx=None, what: str = "") -> None:
    if rc != NF_OK:
        msg = load().nf_last_error(ctx).decode(errors="replace")
        raise NFError(rc, f"{what}: {msg}" if what else msg)
