"""ctypes declarations of libsnap.so (include/snap.h).  Argument marshalling only."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnap.so")
# the diagnostic build (-DSNAP_BOUNDS_CHECK), loaded instead when SNAP_BOUNDS_CHECK=1
LIB_BC_PATH = os.path.join(HERE, "libsnap_bc.so")

SNAP_OK = 0
NOALLOC_SCRATCH_BYTES = 8388608
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "NO_MEMORY",
                5: "WORKSPACE", 6: "NOT_READY"}
FAMILY_A, FAMILY_B, FAMILY_C, FAMILY_TOY, FAMILY_D, FAMILY_E, FAMILY_F = 0, 1, 2, 3, 4, 5, 6
ROW_IC, ROW_MASS, ROW_ENERGY, ROW_BOUNDARY = 1, 2, 4, 8
PATH_AUTO, PATH_GENERAL, PATH_MOMENT, PATH_MIXED = 0, 1, 2, 3
SAMPLE_STATUS = {0: "OK", 1: "MAXITER", 2: "LINESEARCH", 3: "NONFINITE", 4: "INFEASIBLE_PARAMS",
                 5: "RESIDUAL", 6: "SINGULAR", 7: "NOT_MINIMUM", 8: "DEVICE_WAIT"}


class ProblemDesc(C.Structure):
    _fields_ = [("family", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nt", C.c_int),
                ("rows", C.c_uint), ("energy_floor", C.c_double), ("max_batch", C.c_int),
                ("n_flux", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_vars", C.c_int), ("n_rows_nominal", C.c_int), ("n_rows_active", C.c_int),
                ("n_params", C.c_int), ("pattern_nnz", C.c_longlong), ("n_blocks", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("backtracks", C.c_int), ("status", C.c_int),
                ("corrections", C.c_int), ("h_inf", C.c_double), ("kkt_inf", C.c_double),
                ("obj", C.c_double)]


class Options(C.Structure):
    _fields_ = [("tol_kkt", C.c_double), ("tol_h", C.c_double), ("max_iter", C.c_int),
                ("max_backtracks", C.c_int), ("armijo_c1", C.c_double), ("delta0", C.c_double),
                ("max_corrections", C.c_int), ("path", C.c_int), ("w_keep", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int), ("order", C.c_int), ("pack_1d", C.c_int),
                ("sort_1d", C.c_int), ("tile_1d", C.c_int), ("lanes_1d", C.c_int)]


assert C.sizeof(Stats) == 40
assert C.sizeof(ProblemDesc) == 40

_lib = None

# name -> (restype, argtypes)
_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
_PROTOS = {
    "snap_last_error": (C.c_char_p, []),
    "snap_bounds_error": (C.c_int, [C.POINTER(C.c_ulonglong), C.c_int]),
    "snap_version": (C.c_char_p, []),
    "snap_options_default": (C.c_int, [C.POINTER(Options)]),
    "snap_problem_create": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(_vp)]),
    "snap_problem_destroy": (None, [_vp]),
    "snap_problem_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "snap_problem_pattern": (C.c_int, [_vp, _ip, _ip]),
    "snap_problem_active_rows": (C.c_int, [_vp, C.POINTER(C.c_uint8)]),
    "snap_workspace_size": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_size_t)]),
    "snap_project": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                               C.POINTER(Options), _vp, C.c_size_t, _vp]),
    "snap_project_backward": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                        _vp, C.c_size_t, _vp]),
    "snap_constraint_residual": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "snap_pcfm_workspace_size": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_size_t)]),
    "snap_pcfm_sample": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp,
                                   _vp, C.POINTER(Options), _vp, C.c_size_t, _vp]),
    "snap_project_noalloc": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.POINTER(Options), _vp]),
    "snap_batch_create": (C.c_int, [C.c_int, C.POINTER(_vp), C.c_int, _ip, C.POINTER(_vp)]),
    "snap_batch_destroy": (None, [_vp]),
    "snap_batch_bind": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                  C.POINTER(_vp), C.POINTER(_vp)]),
    "snap_batch_workspace_size": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "snap_batch_project": (C.c_int, [_vp, C.POINTER(Options), _vp, _vp, C.c_size_t, _vp]),
    "snap_batch_project_grouped": (C.c_int, [_vp, C.POINTER(Options), _vp, C.c_size_t, _vp]),
    "snap_batch_get_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "snap_batch_get_group_lanes": (C.c_int, [_vp, _ip]),
    "snap_batch_set_group_lanes": (C.c_int, [_vp, _ip]),
    "snap_batch_set_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "snap_batch_autotune": (C.c_int, [_vp, C.POINTER(Options), _vp, C.c_size_t, _vp, C.c_int,
                                      C.POINTER(Schedule), _dp]),
    "snap_batch_capture_graph": (C.c_int, [_vp, C.POINTER(Options), _vp, _vp, C.c_size_t]),
    "snap_batch_launch_graph": (C.c_int, [_vp, _vp]),
    "snap_batch_info": (C.c_int, [_vp, _ip, _ip, _ip]),
    "snap_batch_bind_backward": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
    "snap_batch_project_backward": (C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    "snap_batch_project_backward_grouped": (C.c_int, [_vp, _vp, C.c_size_t, _vp]),
    "snap_batch_capture_graph_backward": (C.c_int, [_vp, _vp, C.c_size_t]),
    "snap_batch_launch_graph_backward": (C.c_int, [_vp, _vp]),
    "snap_measure_fp64_rate": (C.c_int, [C.c_int, _dp]),
    "snap_last_launch_count": (C.c_int, []),
    "snap_profile_enable": (C.c_int, [C.c_int]),
    "snap_profile_reset": (C.c_int, []),
    "snap_profile_read": (C.c_int, [C.c_char_p, _dp, C.POINTER(C.c_longlong)]),
}


def declared_symbols():
    return sorted(_PROTOS)


class SnapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"snap error {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libsnap.so (libsnap_bc.so, the bounds-checked build, when the environment sets
    SNAP_BOUNDS_CHECK=1); raises if that library has not been built (no fallback)."""
    global _lib
    if _lib is None:
        path = LIB_BC_PATH if os.environ.get("SNAP_BOUNDS_CHECK") == "1" else LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"{os.path.basename(path)} not built ({path}); run "
                              "python -m paper_2607_00095_b300.build or __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != SNAP_OK:
        raise SnapError(code, lib().snap_last_error().decode())
    return code
