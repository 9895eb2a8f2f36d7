"""ctypes binding of the C ABI in include/afem_mctdhf.h (argument marshalling only).

The shared library is built in-tree by ``paper_2301_02387_gb300.build`` and
loaded from ``paper_2301_02387_gb300/_lib/libafem.so``.  Loading fails loudly
if it is missing: there is no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libafem.so")

AFEM_OK = 0
AFEM_EINVAL = 1
AFEM_ENOMEM = 2
AFEM_ECUDA = 3
AFEM_EMESH = 4
AFEM_ECG_MAXIT = 5
AFEM_EBREAKDOWN = 6
AFEM_ESINGULAR = 7
AFEM_ENAN = 8
MAX_NUCLEI = 8

MESH_HOST_ONLY = 1

OP_H1 = 0
OP_STIFF = 1
OP_STIFF_F32 = 2
OP_H1_C64 = 3
OP_POS = 4
OP_FORCE = 5
OP_H1_VG = 6
OP_H1_VG_C64 = 7
GAUGE_LENGTH = 0
GAUGE_VELOCITY = 1

CONVERT_F64_F32 = 0
CONVERT_F32_F64 = 1

PROF_GS = 0
PROF_GCELL32 = 1
PROF_STIFF32 = 2
PROF_CGVEC32 = 3
PROF_CELL64 = 4
PROF_COUNT = 5


class MeshDesc(ctypes.Structure):
    _fields_ = [
        ("lo", ctypes.c_double), ("hi", ctypes.c_double),
        ("n_coarse", ctypes.c_int32), ("degree", ctypes.c_int32),
        ("n_nuclei", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("nuc_pos", (ctypes.c_double * 3) * MAX_NUCLEI),
        ("nuc_charge", ctypes.c_double * MAX_NUCLEI),
        ("nuc_levels", ctypes.c_int32 * MAX_NUCLEI),
        ("refine_c", ctypes.c_double),
        ("refine_mode", ctypes.c_int32), ("kelly_max_level", ctypes.c_int32),
        ("kelly_threshold", ctypes.c_double),
    ]


class MeshInfo(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int64), ("n_masters", ctypes.c_int64),
        ("n_interior", ctypes.c_int64), ("n_hanging", ctypes.c_int64),
        ("n_constraint_entries", ctypes.c_int64),
        ("degree", ctypes.c_int32), ("max_level", ctypes.c_int32),
        ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double), ("arnoldi_err", ctypes.c_double),
        ("cg_relres_max", ctypes.c_double),
        ("krylov_m_used", ctypes.c_int32), ("breakdown", ctypes.c_int32),
        ("cg_iters", ctypes.c_int32), ("krylov_substeps", ctypes.c_int32),
        ("dipole", ctypes.c_double * 3),
        ("krylov_dim_sum", ctypes.c_int32), ("krylov_unmet", ctypes.c_int32),
    ]


BATCH_MAX = 256
BATCH_GRAPH = 1
BATCH_MAX_CAND = 8


class BatchTuning(ctypes.Structure):
    _fields_ = [
        ("tuned", ctypes.c_int32), ("block", ctypes.c_int32), ("grid", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32), ("n_candidates", ctypes.c_int32), ("count", ctypes.c_int32),
        ("total_cells", ctypes.c_int64),
        ("cand_ms", ctypes.c_double * BATCH_MAX_CAND),
        ("cand_block", ctypes.c_int32 * BATCH_MAX_CAND),
        ("cand_grid", ctypes.c_int32 * BATCH_MAX_CAND),
    ]


class AfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"afem error {code}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes); every symbol include/afem_mctdhf.h declares
_P = ctypes.c_void_p
SIGNATURES = {
    "afem_last_error": (ctypes.c_char_p, []),
    "afem_kernel_launch_count": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "afem_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "afem_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int]),
    "afem_mesh_create": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.POINTER(_P)]),
    "afem_mesh_create_ex": (ctypes.c_int, [ctypes.POINTER(MeshDesc), ctypes.c_int, ctypes.POINTER(_P)]),
    "afem_mesh_destroy": (ctypes.c_int, [_P]),
    "afem_mesh_get_info": (ctypes.c_int, [_P, ctypes.POINTER(MeshInfo)]),
    "afem_mesh_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "afem_mesh_set_ecs": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "afem_mesh_tables": (ctypes.c_int, [_P, _P, _P, _P]),
    "afem_op_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P]),
    "afem_poisson_batch": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _P, _P, _P]),
    "afem_poisson_batch_ex": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "afem_poisson_boundary_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "afem_two_electron_integrals": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, ctypes.c_int, _P]),
    "afem_batch_stepper_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "afem_batch_stepper_destroy": (ctypes.c_int, [_P]),
    "afem_batch_stepper_step": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               _P, _P]),
    "afem_batch_stepper_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                 _P, _P]),
    "afem_arnoldi_step_ex": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, _P, _P, _P, _P, _P]),
    "afem_mctdhf_set_precision": (ctypes.c_int, [_P, ctypes.c_int]),
    "afem_mctdhf_set_krylov_tol": (ctypes.c_int, [_P, ctypes.c_double]),
    "afem_mctdhf_set_krylov_adaptive": (ctypes.c_int, [_P, ctypes.c_int]),
    "afem_mctdhf_set_imaginary": (ctypes.c_int, [_P, ctypes.c_int]),
    "afem_mctdhf_set_gauge": (ctypes.c_int, [_P, ctypes.c_int]),
    "afem_arnoldi_adaptive": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P, _P, _P, _P]),
    "afem_arnoldi_propagate": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_double, _P, _P, _P, _P]),
    "afem_arnoldi_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P,
                                         _P, _P, _P, _P]),
    "afem_mctdhf_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_P)]),
    "afem_mctdhf_destroy": (ctypes.c_int, [_P]),
    "afem_mctdhf_ci_dim": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "afem_mctdhf_step": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(StepInfo), _P]),
    "afem_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "afem_batch_destroy": (ctypes.c_int, [_P]),
    "afem_batch_op_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int, _P]),
    "afem_batch_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(BatchTuning)]),
    "afem_convert": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, _P]),
    "afem_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _P]),
    "afem_tdse_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                         ctypes.c_int, _P]),
    "afem_tdse_jvp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "afem_tdse_vjp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P, _P]),
}


def load(path=LIB_PATH):
    """Load the shared library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc):
    if rc != AFEM_OK:
        msg = load().afem_last_error().decode(errors="replace")
        raise AfemError(rc, msg)
    return rc
