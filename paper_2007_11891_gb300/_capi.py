"""ctypes binding of the C ABI in include/hdg.h (argument marshalling only).

The shared library is built in-tree by ``paper_2007_11891_gb300.build``.  If
it is missing, every entry point raises: there is no CPU fallback.
"""
import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libhdg_gb300.so")

HDG_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "SINGULAR", 3: "CUDA", 4: "OOM",
                5: "NOT_CONVERGED", 6: "BREAKDOWN", 7: "UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
BASIS = {"nodal": 0, "transformed": 1}

EXPORTED = ["hdg_setup", "hdg_destroy", "hdg_trace_size", "hdg_volume_size", "hdg_boundary_size",
            "hdg_get_nodes", "hdg_apply", "hdg_apply_static", "hdg_solve", "hdg_solve_adjoint", "hdg_last_error",
            "hdg_status_string", "hdg_profile", "hdg_profile_read", "hdg_set_x1_segment", "hdg_set_dz_mode",
            "hdg_set_slots_per_cta", "hdg_autotune", "hdg_set_operator_variant",
            "hdg_set_nodal_variant", "hdg_lowdim_setup", "hdg_lowdim_trace_size", "hdg_lowdim_apply",
            "hdg_lowdim_destroy", "hdg_measure_fma_peak", "hdg_set_cg_variant"]


class HdgLowDimMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ne", ctypes.c_int * 2), ("h_grid", ctypes.POINTER(ctypes.c_double) * 2),
                ("bc", ctypes.c_int * 4)]


class HdgMesh(ctypes.Structure):
    _fields_ = [("ne", ctypes.c_int * 3), ("h_grid", ctypes.POINTER(ctypes.c_double) * 3),
                ("bc", ctypes.c_int * 6)]


class HdgOptions(ctypes.Structure):
    _fields_ = [("tau_hat", ctypes.c_double), ("mass_lumped", ctypes.c_int)]


class HdgSolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner", ctypes.c_int), ("inner_tol", ctypes.c_double), ("precond", ctypes.c_int)]


class HdgSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("applies", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {"iterations": self.iterations, "outer": self.outer, "applies": self.applies,
                "rel_residual": self.rel_residual, "status": STATUS_NAMES.get(self.status, self.status)}


class HdgError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhdg_gb300.so is not built; run paper_2007_11891_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, cd, ci, sz = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    pd = ctypes.POINTER(ctypes.c_double)
    L.hdg_setup.argtypes = [ctypes.POINTER(HdgMesh), ci, ctypes.POINTER(HdgOptions), ctypes.POINTER(vp)]
    L.hdg_setup.restype = ci
    L.hdg_destroy.argtypes = [vp]
    L.hdg_destroy.restype = None
    for f in ("hdg_trace_size", "hdg_volume_size", "hdg_boundary_size"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = sz
    L.hdg_get_nodes.argtypes = [vp, pd]
    L.hdg_get_nodes.restype = ci
    L.hdg_apply.argtypes = [vp, ci, pd, ci, ci, vp, vp, vp]
    L.hdg_apply.restype = ci
    L.hdg_apply_static.argtypes = [vp, ci, pd, vp, vp, vp]
    L.hdg_apply_static.restype = ci
    L.hdg_solve.argtypes = [vp, ci, pd, vp, vp, vp, vp, vp, ctypes.POINTER(HdgSolveOpts),
                            ctypes.POINTER(HdgSolveInfo), vp]
    L.hdg_solve.restype = ci
    L.hdg_solve_adjoint.argtypes = [vp, ci, pd, vp, vp, vp, vp, ctypes.POINTER(HdgSolveOpts),
                                    ctypes.POINTER(HdgSolveInfo), vp]
    L.hdg_solve_adjoint.restype = ci
    L.hdg_set_slots_per_cta.argtypes = [vp, ci]
    L.hdg_set_slots_per_cta.restype = ci
    L.hdg_autotune.argtypes = [vp, ci, pd, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), pd, vp]
    L.hdg_autotune.restype = ci
    L.hdg_set_dz_mode.argtypes = [vp, ci]
    L.hdg_set_dz_mode.restype = ci
    L.hdg_set_operator_variant.argtypes = [vp, ci]
    L.hdg_set_operator_variant.restype = ci
    L.hdg_set_cg_variant.argtypes = [vp, ci]
    L.hdg_set_cg_variant.restype = ci
    L.hdg_set_nodal_variant.argtypes = [vp, ci]
    L.hdg_set_nodal_variant.restype = ci
    L.hdg_lowdim_setup.argtypes = [ctypes.POINTER(HdgLowDimMesh), ci, ctypes.POINTER(HdgOptions),
                                   ctypes.POINTER(vp)]
    L.hdg_lowdim_setup.restype = ci
    L.hdg_lowdim_trace_size.argtypes = [vp]
    L.hdg_lowdim_trace_size.restype = ctypes.c_size_t
    L.hdg_lowdim_apply.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ci, vp, vp, vp]
    L.hdg_lowdim_apply.restype = ci
    L.hdg_lowdim_destroy.argtypes = [vp]
    L.hdg_lowdim_destroy.restype = None
    L.hdg_set_x1_segment.argtypes = [vp, ci]
    L.hdg_set_x1_segment.restype = ci
    L.hdg_profile.argtypes = [vp, ci]
    L.hdg_profile.restype = ci
    L.hdg_profile_read.argtypes = [vp, ci, pd, ctypes.POINTER(ctypes.c_longlong)]
    L.hdg_profile_read.restype = ci
    L.hdg_measure_fma_peak.argtypes = [ci, pd, vp]
    L.hdg_measure_fma_peak.restype = ci
    L.hdg_last_error.argtypes = []
    L.hdg_last_error.restype = ctypes.c_char_p
    L.hdg_status_string.argtypes = [ci]
    L.hdg_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status, where):
    if status != HDG_OK:
        raise HdgError(status, where, lib().hdg_last_error().decode())
    return status


def doubles(values):
    arr = (ctypes.c_double * len(values))(*[float(v) for v in values])
    return arr
