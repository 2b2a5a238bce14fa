"""ctypes declarations of the libmto C ABI (include/mto.h).

Argument marshalling only: every step of the solver runs in libmto's CUDA
kernels.  Loading fails loudly when libmto.so has not been built; there is no
fallback implementation.
"""

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmto.so")

STATUS = {
    0: "MTO_OK",
    1: "MTO_ERR_ARG",
    2: "MTO_ERR_UNSUPPORTED_MESH",
    3: "MTO_ERR_OOM",
    4: "MTO_ERR_CUDA",
    5: "MTO_ERR_NOT_CONVERGED",
    6: "MTO_ERR_BREAKDOWN",
    7: "MTO_ERR_TIMEOUT",
    8: "MTO_ERR_STATE",
}
OK, ERR_ARG, ERR_UNSUPPORTED_MESH, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_BREAKDOWN, \
    ERR_TIMEOUT, ERR_STATE = range(9)

EDGE_BOTTOM, EDGE_LEFT, EDGE_RIGHT, EDGE_TOP = 1, 2, 4, 8
COARSE_GALERKIN, COARSE_REDISCRETIZE = 0, 1
PRECISION_FP64, PRECISION_MIXED = 0, 1


class SolverOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_it", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("n_coarsen", ctypes.c_int),
        ("coarse_kind", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("rr_every", ctypes.c_int),
        ("flexible", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("gamma", ctypes.c_int),
        ("concurrent_rhs", ctypes.c_int),
    ]


class SolveStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("rel_res_rec", ctypes.c_double),
        ("rel_res_true", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
        ("ms_solve", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PoissonOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_it", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("n_coarsen", ctypes.c_int),
        ("cluster_ctas", ctypes.c_int),
        ("precision", ctypes.c_int),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("n_phase", ctypes.c_int),
        ("x_dev", ctypes.c_void_p),
        ("E_phase", ctypes.POINTER(ctypes.c_double)),
        ("penal", ctypes.c_double),
        ("n_rhs", ctypes.c_int),
        ("f_dev", ctypes.c_void_p),
        ("u_dev", ctypes.c_void_p),
        ("compliance_dev", ctypes.c_void_p),
        ("dcdx_dev", ctypes.c_void_p),
    ]


class MtoError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the full exported surface of include/mto.h.
SIGNATURES = {
    "mto_default_opts": (None, [ctypes.POINTER(SolverOpts)]),
    "mto_create_mesh": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_uint, ctypes.POINTER(SolverOpts), ctypes.c_int, _P]),
    "mto_set_design": (ctypes.c_int, [_P, ctypes.c_int, _P, _D, ctypes.c_double]),
    "mto_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(SolveStats)]),
    "mto_last_stats": (ctypes.c_int, [_P, ctypes.POINTER(SolveStats)]),
    "mto_compliance_grad": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    "mto_run_host": (ctypes.c_int, [_P, ctypes.c_int, _P, _D, ctypes.c_double, ctypes.c_int, _P, _P,
                                    _P, _P, ctypes.POINTER(SolveStats)]),
    "mto_run_host_async": (ctypes.c_int, [_P, ctypes.c_int, _P, _D, ctypes.c_double, ctypes.c_int, _P, _P,
                                          _P, _P]),
    "mto_run_host_wait": (ctypes.c_int, [_P, ctypes.POINTER(SolveStats)]),
    "mto_apply_operator": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "mto_apply_preconditioner": (ctypes.c_int, [_P, _P, _P]),
    "mto_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mto_get_moduli": (ctypes.c_int, [_P, _P]),
    "mto_compliance_grad_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                   _P, _D, ctypes.c_double, _P, _P, _P, _P, ctypes.c_int,
                                                   _P]),
    "mto_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                        ctypes.POINTER(BatchItem), _P]),
    "mto_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(SolveStats)]),
    "mto_batch_tune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "mto_batch_time": (ctypes.c_int, [_P, _D]),
    "mto_batch_destroy": (None, [_P]),
    "mto_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(BatchItem),
                                         ctypes.POINTER(SolveStats), _P]),
    "mto_autotune": (ctypes.c_int, [_P]),
    "mto_get_launch_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mto_set_launch_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "mto_set_kernel_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "mto_get_kernel_times": (ctypes.c_int, [_P, _D, ctypes.POINTER(ctypes.c_longlong)]),
    "mto_get_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "mto_measure_fp64_rate": (ctypes.c_int, [ctypes.c_int, _P, _D]),
    "mto_poisson_default_opts": (None, [ctypes.POINTER(PoissonOpts)]),
    "mto_poisson_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(PoissonOpts), ctypes.c_int, _P]),
    "mto_poisson_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(SolveStats)]),
    "mto_poisson_apply_operator": (ctypes.c_int, [_P, _P, _P]),
    "mto_poisson_apply_preconditioner": (ctypes.c_int, [_P, _P, _P]),
    "mto_poisson_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
    "mto_poisson_destroy": (None, [_P]),
    "mto_set_device_memory_limit": (None, [ctypes.c_size_t]),
    "mto_device_memory_in_use": (ctypes.c_size_t, []),
    "mto_destroy": (None, [_P]),
    "mto_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mto_cuda_error_string": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libmto.so (built in-tree by paper_2301_07457_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libmto.so not found at {LIB_PATH}; build it first with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code, where):
    if code != OK:
        if code == ERR_CUDA and _lib is not None:
            where = f"{where} ({_lib.mto_cuda_error_string().decode()})"
        raise MtoError(code, where)


def default_opts():
    o = SolverOpts()
    load().mto_default_opts(ctypes.byref(o))
    return o
