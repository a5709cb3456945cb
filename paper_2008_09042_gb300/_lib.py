"""ctypes binding of libmpi_gb300.so (argument marshalling only).

The library must exist: there is no fallback implementation.  Build it with
``python -m paper_2008_09042_gb300.build``.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpi_gb300.so")

MPI_OK = 0
STATUS_NAMES = {0: "MPI_OK", 1: "MPI_ERR_ARG", 2: "MPI_ERR_SHAPE", 3: "MPI_ERR_CUDA", 4: "MPI_ERR_OOM",
                5: "MPI_ERR_NOT_CONVERGED", 6: "MPI_ERR_TIMEOUT", 7: "MPI_ERR_UNSUPPORTED"}

TRAJ_CARTESIAN = 0
TRAJ_RADIAL = 1
PREC = {"fp32": 0, "bf16": 1, "fp32_simt": 2, "mixed": 3}

# Every symbol include/mpi_gb300.h declares.
EXPORTS = [
    "mpi_ctx_create", "mpi_ctx_destroy", "mpi_ctx_set_stream", "mpi_ctx_synchronize", "mpi_ctx_reserve",
    "mpi_last_error", "mpi_ctx_launch_count", "mpi_ctx_workspace_bytes", "mpi_ctx_set_autotune", "mpi_ctx_set_line_kernel", "mpi_ctx_set_wait_limit", "mpi_ctx_inject_stall", "mpi_ctx_tuning_record", "mpi_ctx_profile", "mpi_ctx_profile_read", "mpi_ctx_profile_kernel", "mpi_plan_create", "mpi_plan_destroy", "mpi_plan_grid_index",
    "mpi_basis_load_dense", "mpi_basis_load_tucker", "mpi_basis_destroy", "mpi_basis_expand", "mpi_forward", "mpi_adjoint",
    "mpi_jacobian", "mpi_jacobian_adjoint", "mpi_basis_project", "mpi_sm_estimate", "mpi_image_solve",
    "mpi_tv_prox", "mpi_forward_noalloc", "mpi_batch_create", "mpi_batch_run", "mpi_batch_kernel_count",
    "mpi_batch_destroy", "mpi_expand_path", "mpi_forward_host", "mpi_adjoint_host", "mpi_maxwell_basis_2d",
    "mpi_forward_maps", "mpi_adjoint_maps", "mpi_jacobian_maps", "mpi_jacobian_adjoint_maps", "mpi_sm_estimate_maps",
    "mpi_maxwell_basis_3d", "mpi_tucker_compress", "mpi_image_solve_dynamic",
    "mpi_batch_group_count", "mpi_ctx_tf32_reading", "mpi_ctx_set_tf32x3",
]


class MpiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("dims", ctypes.c_int * 3),
        ("kind", ctypes.c_int),
        ("M", ctypes.c_int),
        ("sample_idx", ctypes.c_void_p),
        ("traj", ctypes.c_void_p),
        ("kb_width", ctypes.c_int),
        ("oversamp", ctypes.c_float),
    ]


class BatchSlice(ctypes.Structure):
    _fields_ = [
        ("plan", ctypes.c_void_p), ("basis", ctypes.c_void_p), ("C", ctypes.c_int),
        ("alpha", ctypes.c_void_p), ("p", ctypes.c_void_p), ("y", ctypes.c_void_p), ("x", ctypes.c_void_p),
    ]


class IrgnParams(ctypes.Structure):
    _fields_ = [
        ("n_outer", ctypes.c_int), ("n_cg", ctypes.c_int),
        ("a0", ctypes.c_double), ("b0", ctypes.c_double), ("decay", ctypes.c_double),
        ("floor_", ctypes.c_double), ("gamma", ctypes.c_double), ("scale_target", ctypes.c_double),
    ]


class AdmmParams(ctypes.Structure):
    _fields_ = [
        ("n_outer", ctypes.c_int), ("n_cg", ctypes.c_int), ("n_tv", ctypes.c_int),
        ("rho0", ctypes.c_double), ("mu", ctypes.c_double), ("tau", ctypes.c_double),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load the library (once) and declare argument types."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with python -m paper_2008_09042_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mpi_ctx_create": [pp, i, vp],
        "mpi_ctx_destroy": [vp],
        "mpi_ctx_set_stream": [vp, vp],
        "mpi_ctx_synchronize": [vp],
        "mpi_ctx_reserve": [vp, vp, vp, i],
        "mpi_ctx_set_autotune": [vp, i],
        "mpi_ctx_set_line_kernel": [vp, i],
        "mpi_ctx_set_wait_limit": [vp, i64],
        "mpi_ctx_inject_stall": [vp, i],
        "mpi_ctx_set_tf32x3": [vp, i],
        "mpi_ctx_tuning_record": [vp, i, ctypes.POINTER(ctypes.c_char_p)],
        "mpi_ctx_profile": [vp, i],
        "mpi_ctx_profile_read": [vp, i, ctypes.POINTER(d), ctypes.POINTER(i64), i],
        "mpi_ctx_profile_kernel": [vp, i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(d), ctypes.POINTER(i64)],
        "mpi_plan_create": [vp, ctypes.POINTER(PlanDesc), pp],
        "mpi_plan_destroy": [vp],
        "mpi_plan_grid_index": [vp, vp, vp],
        "mpi_basis_load_dense": [vp, vp, i, i, i, pp],
        "mpi_basis_load_tucker": [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  i, i, pp],
        "mpi_basis_destroy": [vp],
        "mpi_maxwell_basis_2d": [vp, i, i, d, d, d, vp, i, vp, i, i, vp, vp],
        "mpi_maxwell_basis_3d": [vp, i, i, i, d, d, d, d, vp, i, vp, i, i, vp, vp],
        "mpi_tucker_compress": [vp, vp, ctypes.POINTER(ctypes.c_int), i, d, pp, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(d)],
        "mpi_expand_path": [vp, i, i, i],
        "mpi_basis_expand": [vp, vp, vp, i, vp, i],
        "mpi_forward": [vp, vp, vp, vp, i, vp, vp, i],
        "mpi_adjoint": [vp, vp, vp, vp, i, vp, vp, i],
        "mpi_forward_host": [vp, vp, vp, vp, i, vp, vp, i],
        "mpi_adjoint_host": [vp, vp, vp, vp, i, vp, vp, i],
        "mpi_jacobian": [vp, vp, vp, vp, i, vp, vp, vp, vp, i],
        "mpi_jacobian_adjoint": [vp, vp, vp, vp, i, vp, vp, vp, vp, i],
        "mpi_basis_project": [vp, vp, vp, i, vp],
        "mpi_sm_estimate": [vp, vp, vp, vp, i, ctypes.POINTER(IrgnParams), vp, vp, vp, i],
        "mpi_forward_maps": [vp, vp, vp, i, vp, i, vp, vp, i],
        "mpi_adjoint_maps": [vp, vp, vp, i, vp, i, vp, vp, i],
        "mpi_jacobian_maps": [vp, vp, vp, i, vp, i, vp, vp, vp, vp, i],
        "mpi_jacobian_adjoint_maps": [vp, vp, vp, i, vp, i, vp, vp, vp, vp, i],
        "mpi_sm_estimate_maps": [vp, vp, vp, i, vp, i, ctypes.POINTER(IrgnParams), vp, vp, vp, i],
        "mpi_image_solve": [vp, vp, vp, vp, i, vp, vp, ctypes.POINTER(AdmmParams), vp, vp, i],
        "mpi_image_solve_dynamic": [vp, ctypes.POINTER(ctypes.c_void_p), i, vp, vp, i, vp, vp,
                                    ctypes.POINTER(AdmmParams), vp, vp, i],
        "mpi_tv_prox": [vp, vp, vp, d, i, vp],
        "mpi_forward_noalloc": [vp, vp, vp, vp, i, vp, vp],
        "mpi_batch_create": [vp, ctypes.POINTER(BatchSlice), i, i, i, pp],
        "mpi_batch_run": [vp, vp],
        "mpi_batch_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.mpi_last_error.argtypes = [vp]
    lib.mpi_last_error.restype = ctypes.c_char_p
    lib.mpi_ctx_launch_count.argtypes = [vp]
    lib.mpi_ctx_launch_count.restype = i64
    lib.mpi_ctx_workspace_bytes.argtypes = [vp]
    lib.mpi_ctx_workspace_bytes.restype = i64
    lib.mpi_batch_kernel_count.argtypes = [vp]
    lib.mpi_batch_kernel_count.restype = i64
    lib.mpi_batch_group_count.argtypes = [vp]
    lib.mpi_batch_group_count.restype = i
    lib.mpi_ctx_tf32_reading.argtypes = [vp]
    lib.mpi_ctx_tf32_reading.restype = i
    _lib = lib
    return lib


def check(ctx_handle, status):
    if status != MPI_OK:
        msg = load().mpi_last_error(ctx_handle) if ctx_handle else b""
        raise MpiError(status, (msg or b"").decode(errors="replace"))
