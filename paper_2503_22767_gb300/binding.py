"""ctypes binding of the C ABI in ``include/mpm.h`` (argument marshalling only).

Every entry point keeps its C name.  The library is the CUDA build in
``_build/libmpm.so``; importing this module builds it if it is missing and
raises if that fails -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

c_int, c_double, c_void_p, c_longlong = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
P_float = ctypes.POINTER(ctypes.c_float)
P_int = ctypes.POINTER(ctypes.c_int)

MPM_OK, MPM_ERR_ARG, MPM_ERR_CUDA, MPM_ERR_OOM = 0, -1, -2, -3
MPM_ERR_STATE, MPM_ERR_NUMERIC, MPM_ERR_DOMAIN, MPM_ERR_TIMEOUT = -4, -5, -6, -7
MPM_OPT_TIMING, MPM_OPT_BLOCK, MPM_OPT_FUSE_GRID, MPM_OPT_GRAPHS, MPM_OPT_STREAMS = 1, 2, 3, 4, 6
MPM_OPT_PDL = 7
MPM_OPT_ADJOINT_BLOCKS = 8
MPM_OPT_GRID_BLOCKS = 10
MPM_OPT_PERSISTENT = 11
MPM_OPT_SPIN_LIMIT = 12
MPM_OPT_SCATTER_2D = 13
MPM_OPT_RESIDENT_SEGMENTS = 14
MPM_OPT_SEGMENT_BYTES = 15
STATUS_NAMES = {0: "MPM_OK", -1: "MPM_ERR_ARG", -2: "MPM_ERR_CUDA", -3: "MPM_ERR_OOM",
                -4: "MPM_ERR_STATE", -5: "MPM_ERR_NUMERIC", -6: "MPM_ERR_DOMAIN",
                -7: "MPM_ERR_TIMEOUT"}

#: every function the header declares (checked by the tests)
EXPORTS = ["mpm_create", "mpm_destroy", "mpm_last_error", "mpm_forward", "mpm_backward",
           "mpm_forward_host", "mpm_backward_host", "mpm_read_state", "mpm_read_state_strain",
           "mpm_sort_particles",
           "mpm_set_option", "mpm_get_option", "mpm_autotune", "mpm_get_stats", "mpm_reset_stats",
           "mpm_substep_noalloc", "mpm_noalloc_last_error", "mpm_set_boundaries", "mpm_set_field_gradient", "mpm_field_gradient_grad",
           # design maps and optimiser step (mpm_design.h)
           "mpm_design_create", "mpm_design_destroy", "mpm_design_last_error", "mpm_design_forward",
           "mpm_design_backward", "mpm_adam_step"]
MPM_NOALLOC_MAX_NODES = 262144


MPM_MAX_BOUNDARIES = 8
MPM_BOUNDARY_COULOMB, MPM_BOUNDARY_NONSLIP, MPM_BOUNDARY_ATTACHED = 0, 1, 2


class mpm_boundary(ctypes.Structure):
    """Mirror of mpm_boundary (include/mpm.h)."""
    _fields_ = [("kind", c_int), ("mu", ctypes.c_float), ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class mpm_design_config(ctypes.Structure):
    """Mirror of mpm_design_config (include/mpm_design.h)."""
    _fields_ = [("dim", c_int), ("n_particles", c_int), ("n_regions", c_int), ("n_tasks", c_int),
                ("n_steps", c_int), ("dt", ctypes.c_double), ("filter_radius", ctypes.c_double),
                ("Br_max", ctypes.c_double), ("B_max", ctypes.c_double), ("f_min", ctypes.c_double),
                ("f_max", ctypes.c_double), ("delta", ctypes.c_double)]


class mpm_config(ctypes.Structure):
    _fields_ = [
        ("dim", c_int), ("grid_res", c_int), ("dt", c_double), ("n_steps", c_int),
        ("n_instances", c_int), ("n_particles", P_int), ("n_designs", c_int),
        ("design_of_instance", P_int), ("E", c_double), ("nu", c_double), ("rho0", c_double),
        ("p_vol", c_double), ("simp_eps", c_double), ("simp_q", c_int), ("damping_c", c_double),
        ("gravity", c_double * 3), ("bound", c_int), ("wall_mode", c_int), ("floor_mu", c_double),
        ("loss_kind", c_int), ("checkpoint_every", c_int),
    ]


class mpm_stats(ctypes.Structure):
    _fields_ = [("launches", c_longlong), ("timed_launches", c_longlong * 4),
                ("timed_ms", c_double * 4), ("timed_bytes", c_double * 4),
                ("device_bytes", c_longlong), ("class_launches", c_longlong * 4)]


class MpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from . import build
    return build.LIB


def load():
    """Load (building first if needed) the CUDA library and declare signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build
        path = build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing and could not be built")
        lib = ctypes.CDLL(path)
        pf, pi, vp = P_float, P_int, c_void_p
        H = c_void_p
        sig = {
            "mpm_create": ([ctypes.POINTER(mpm_config), ctypes.POINTER(c_void_p)], c_int),
            "mpm_destroy": ([H], c_int),
            "mpm_last_error": ([H], ctypes.c_char_p),
            "mpm_forward": ([H, pf, pf, pf, pf, pf, pf, pf, pf, vp], c_int),
            "mpm_backward": ([H, pf, pf, pf, pf, vp], c_int),
            "mpm_forward_host": ([H, pf, pf, pf, pf, pf, pf, pf, pf, vp], c_int),
            "mpm_backward_host": ([H, pf, pf, pf, pf, vp], c_int),
            "mpm_read_state": ([H, pf, pf, pf, pf, vp], c_int),
            "mpm_read_state_strain": ([H, pf, pf, pf, pf, vp], c_int),
            "mpm_sort_particles": ([H, pf, pi, pi, vp], c_int),
            "mpm_set_option": ([H, c_int, c_longlong], c_int),
            "mpm_get_option": ([H, c_int, ctypes.POINTER(c_longlong)], c_int),
            "mpm_autotune": ([H, ctypes.c_char_p, c_int, vp], c_int),
            "mpm_get_stats": ([H, ctypes.POINTER(mpm_stats)], c_int),
            "mpm_reset_stats": ([H], c_int),
            "mpm_substep_noalloc": ([ctypes.POINTER(mpm_config), c_int, pf, pf, pf, pf, pf, vp], c_int),
            "mpm_noalloc_last_error": ([], ctypes.c_char_p),
            "mpm_set_boundaries": ([H, c_int, ctypes.POINTER(mpm_boundary), pf, vp], c_int),
            "mpm_set_field_gradient": ([H, pf, vp], c_int),
            "mpm_field_gradient_grad": ([H, pf, vp], c_int),
            "mpm_design_create": ([ctypes.POINTER(mpm_design_config), pf, pi, ctypes.POINTER(c_void_p), vp],
                                  c_int),
            "mpm_design_destroy": ([H], c_int),
            "mpm_design_last_error": ([H], ctypes.c_char_p),
            "mpm_design_forward": ([H, ctypes.c_float, pf, pf, pf, pf, pf, pf, pf, pf, pf, vp], c_int),
            "mpm_design_backward": ([H, pf, pf, pf, pf, pf, pf, pf, pf, pf, vp], c_int),
            "mpm_adam_step": ([c_longlong, pf, pf, pf, pf, c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp], c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def fptr(t):
    """float* of a torch tensor / numpy array / raw int address (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.cast(t, P_float)
    if hasattr(t, "data_ptr"):
        return ctypes.cast(t.data_ptr(), P_float)
    return t.ctypes.data_as(P_float)


def iptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.cast(t.data_ptr(), P_int)
    return t.ctypes.data_as(P_int)


def check(lib, handle, status, what):
    if status != MPM_OK:
        msg = lib.mpm_last_error(handle) if handle else b""
        raise MpmError(status, f"{what}: {msg.decode() if msg else ''}")
