"""ctypes loader of ``libfmpb.so`` (argument marshalling only).

The library is built in-tree by ``paper_2201_12050_gb300.build``.  There is
no fallback: if the shared library is missing or cannot be loaded, every
entry point raises ``FmpbLibraryMissing``.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmpb.so")

STATUS = {0: "FMPB_OK", -1: "FMPB_EINVAL", -2: "FMPB_ENOMEM", -3: "FMPB_EMESH", -4: "FMPB_EADMISS",
          -5: "FMPB_ENOCONV", -6: "FMPB_ETIMEOUT", -7: "FMPB_ENAN", -8: "FMPB_ECUDA"}


class FmpbLibraryMissing(ImportError):
    pass


class FmpbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Lattice(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_int32 * 3), ("vectors", (ctypes.c_double * 3) * 3)]


class OperatorOpts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("n_t", ctypes.c_int), ("precision", ctypes.c_int),
                ("beta_re", ctypes.c_double), ("beta_im", ctypes.c_double),
                ("halfspace", ctypes.c_int32), ("plane_axis", ctypes.c_int32), ("plane_offset", ctypes.c_double),
                ("Rp_re", ctypes.c_double), ("Rp_im", ctypes.c_double),
                ("n_t_near", ctypes.c_int32), ("near_levels", ctypes.c_int32), ("element", ctypes.c_int32),
                ("pressure_order", ctypes.c_int32), ("n_t_rule_err", ctypes.c_double)]


class C64(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class Incident(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("vec", ctypes.c_double * 3), ("amp", C64)]


class OperatorInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("N", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("form", ctypes.c_int32), ("n_t", ctypes.c_int32), ("B", ctypes.c_int64),
                ("P", ctypes.c_int32 * 3), ("F", ctypes.c_int64), ("n_near", ctypes.c_int32),
                ("bytes_device", ctypes.c_size_t), ("precision", ctypes.c_int32),
                ("beta_re", ctypes.c_double), ("beta_im", ctypes.c_double),
                ("halfspace", ctypes.c_int32), ("hankel_axis", ctypes.c_int32), ("n_near_image", ctypes.c_int32),
                ("image_separate", ctypes.c_int32), ("near_levels", ctypes.c_int32),
                ("n_m2l_near", ctypes.c_int64), ("n_p2p_near", ctypes.c_int64), ("element", ctypes.c_int32),
                ("pressure_order", ctypes.c_int32), ("n_t_rule_err", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("timeout_ms", ctypes.c_int), ("inner_tol", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("relres_est", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("refinements", ctypes.c_int)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_rhs", ctypes.c_int), ("cache_entries", ctypes.c_int),
                ("precision", ctypes.c_int), ("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("nv", ctypes.c_int64), ("tris", ctypes.c_void_p), ("ntri", ctypes.c_int64),
                ("lattice", Lattice), ("k", ctypes.c_double), ("form", ctypes.c_int), ("n_t", ctypes.c_int),
                ("R", ctypes.c_int), ("dirs", ctypes.c_void_p), ("amps", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("R", ctypes.c_int), ("iters_max", ctypes.c_int),
                ("relres_true_max", ctypes.c_double), ("cache_hit", ctypes.c_int), ("batched_with", ctypes.c_int),
                ("queue_ms", ctypes.c_double), ("build_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cache_hits", ctypes.c_int64), ("batches", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("hbm_in_use", ctypes.c_size_t), ("hbm_high_water", ctypes.c_size_t)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double
INT = ctypes.c_int

# name -> (restype, argtypes); the entry points declared in include/fmpb.h
SIGNATURES = {
    "fmpb_last_error": (ctypes.c_char_p, []),
    "fmpb_version": (INT, []),
    "fmpb_operator_create": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), D, ctypes.POINTER(OperatorOpts), P,
                                   ctypes.POINTER(P)]),
    "fmpb_operator_get_info": (INT, [P, ctypes.POINTER(OperatorInfo)]),
    "fmpb_operator_destroy": (None, [P]),
    "fmpb_rhs_plane_wave": (INT, [P, INT, P, P, P, P]),
    "fmpb_matvec": (INT, [P, INT, P, P, P]),
    "fmpb_solve": (INT, [P, INT, P, P, ctypes.POINTER(SolveOpts), P, P]),
    "fmpb_solve_batch": (INT, [P, INT, INT, P, P, ctypes.POINTER(SolveOpts), P, P]),
    "fmpb_operator_check": (INT, [P, P]),
    "fmpb_field": (INT, [P, INT, P, P, P, I64, P, P, P]),
    "fmpb_build_blocks": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), D, INT, P, P, P]),
    "fmpb_multipole_tables": (INT, [P, I64, P, I64, D, INT, P, P, P]),
    "fmpb_rhs_incident": (INT, [P, INT, P, P, P]),
    "fmpb_insertion_loss": (INT, [P, INT, P, P, I64, P, P, P]),
    "fmpb_halfspace_plan": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), INT, D, P, P, P]),
    "fmpb_halfspace_plan_q9": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), INT, D, P, P, P]),
    "fmpb_near2_plan_counts": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), INT, INT, P, P, P, P]),
    "fmpb_near2_plan_counts_q9": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), INT, INT, P, P, P, P]),
    "fmpb_field_incident": (INT, [P, INT, P, P, I64, P, P, P]),
    "fmpb_build_blocks_admittance": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), D, D, D, INT, P, P, P]),
    "fmpb_multipole_tables_admittance": (INT, [P, I64, P, I64, D, D, D, INT, P, P, P]),
    "fmpb_build_blocks_q9": (INT, [P, I64, P, I64, ctypes.POINTER(Lattice), D, D, D, INT, P, P, P]),
    "fmpb_build_blocks_q9p": (INT, [P, I64, P, I64, INT, ctypes.POINTER(Lattice), D, D, D, INT, P, P, P]),
    "fmpb_m2l_blocks": (INT, [D, INT, INT, P, P, P]),
    "fmpb_offset_gemm_bf16": (INT, [P, INT, P, I64, I64, P, INT, P, P, INT, P]),
    "fmpb_offset_gemm2_bf16": (INT, [P, INT, P, I64, I64, P, INT, P, I64, P, P, P, INT, P]),
    "fmpb_circulant_shape": (INT, [P, P, P]),
    "fmpb_circulant_spectrum": (INT, [P, I64, P, P, P]),
    "fmpb_circulant_apply": (INT, [P, I64, P, INT, P, P, INT, P]),
    "fmpb_circulant_apply_static": (INT, [P, I64, P, INT, P, P, INT, P]),
    "fmpb_circulant_apply_bf16": (INT, [P, I64, P, INT, P, P, INT, P]),
    "fmpb_circulant_apply_f32": (INT, [P, I64, P, INT, P, P, INT, P]),
    "fmpb_server_create": (INT, [ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]),
    "fmpb_server_submit": (INT, [P, ctypes.POINTER(Request), P, ctypes.POINTER(ctypes.c_uint64)]),
    "fmpb_server_wait": (INT, [P, ctypes.c_uint64, INT, ctypes.POINTER(Result)]),
    "fmpb_server_get_stats": (INT, [P, ctypes.POINTER(ServerStats)]),
    "fmpb_server_destroy": (None, [P]),
    "fmpb_kernel_launches": (ctypes.c_uint64, []),
    "fmpb_profile_enable": (None, [INT]),
    "fmpb_profile_reset": (INT, []),
    "fmpb_profile_summary": (INT, [ctypes.c_char_p, ctypes.c_size_t]),
    "fmpb_tuning_summary": (INT, [ctypes.c_char_p, ctypes.c_size_t]),
    "fmpb_set_tile_variant": (INT, [INT]),
    "fmpb_set_dft_plan": (INT, [INT]),
}

_lib = None


def lib():
    """The loaded library (loaded once); raises FmpbLibraryMissing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FmpbLibraryMissing(f"{LIB_PATH} is not built; run paper_2201_12050_gb300.build.build()")
    try:
        L = ctypes.CDLL(LIB_PATH)
    except OSError as e:
        raise FmpbLibraryMissing(f"cannot load {LIB_PATH}: {e}") from e
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int):
    if status != 0:
        raise FmpbError(status, lib().fmpb_last_error().decode())
    return status
