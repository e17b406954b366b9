"""ctypes declarations of the C ABI in include/pstd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libpstd.so")

NEUMANN, DIRICHLET, PERIODIC, NEUMANN_MID, DIRICHLET_MID = 0, 1, 2, 3, 4
# wall codes: "Nm" / "Dm" put the right wall at mid-cell, x = (N - 1/2) dx
BC_CODES = {"N": NEUMANN, "D": DIRICHLET, "P": PERIODIC, "Nm": NEUMANN_MID, "Dm": DIRICHLET_MID}
U_HALFSTEP, U_AS_GIVEN = 0, 1
NODES_P, HALF_U, NODES_U, HALF_P = 0, 1, 2, 3
OP_DIFF, OP_INTERP = 0, 1

ERRORS = {0: "PSTD_OK", -1: "PSTD_EINVAL", -2: "PSTD_EUNSTABLE", -3: "PSTD_ENOMEM",
          -4: "PSTD_ECUDA", -5: "PSTD_ETIMEOUT", -6: "PSTD_EUNSUPPORTED"}

# Every symbol include/pstd.h declares, with (restype, argtypes).
SIGNATURES = {
    "pstd_plan": (c_int, [c_void_p, c_void_p, POINTER(c_void_p)]),
    "pstd_plan_ex": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_void_p)]),
    "pstd_plan_autotune": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_void_p), POINTER(c_double)]),
    "pstd_plan_schedule": (c_int, [c_void_p, c_int, POINTER(c_int)]),
    "pstd_plan_persistent": (c_int, [c_void_p, POINTER(c_int)]),
    "pstd_field_shape": (c_int, [c_void_p, c_int, POINTER(c_int64)]),
    "pstd_field_numel": (c_int64, [c_void_p, c_int]),
    "pstd_grad": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "pstd_apply_shape": (c_int, [c_void_p, c_int, c_int, POINTER(c_int64)]),
    "pstd_apply": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "pstd_init_velocity": (c_int, [c_void_p, c_void_p, POINTER(c_void_p)]),
    "pstd_step": (c_int, [c_void_p, c_void_p, POINTER(c_void_p)]),
    "pstd_run": (c_int, [c_void_p, c_void_p, POINTER(c_void_p), c_int64]),
    "pstd_init_prev": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pstd_run2": (c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    "pstd_energy": (c_int, [c_void_p, c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_double)]),
    "pstd_sync": (c_int, [c_void_p]),
    "pstd_free": (c_int, [c_void_p]),
    "pstd_strerror": (c_char_p, [c_int]),
    "pstd_last_cuda_error": (c_char_p, []),
    "pstd_dt_from_cfl": (c_double, [c_double, c_double, c_double]),
    "pstd_last_launch_count": (c_int64, [c_void_p]),
    "pstd_version": (c_char_p, []),
    "pstd_batch_plan": (c_int, [c_void_p, c_int, c_void_p, POINTER(c_void_p)]),
    "pstd_batch_member": (c_int, [c_void_p, c_int, POINTER(c_void_p)]),
    "pstd_batch_init_velocity": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p)]),
    "pstd_batch_run": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), c_int64]),
    "pstd_batch_combine": (c_int, [c_void_p, POINTER(c_double), POINTER(c_void_p), c_void_p]),
    "pstd_batch_free": (c_int, [c_void_p]),
    "pstd_batch_last_launch_count": (c_int64, [c_void_p]),
    "pstd_batch_set_persistent": (c_int, [c_void_p, c_int, ctypes.c_longlong, c_int]),
    "pstd_batch_persistent_kind": (c_int, [c_void_p]),
    "pstd_batch_sync": (c_int, [c_void_p]),
    "pstd_reflection_combos": (c_int, [c_void_p, POINTER(c_double), c_void_p, POINTER(c_double)]),
    "pstd_step_noalloc": (c_int, [c_void_p, c_void_p, POINTER(c_void_p), c_int64, c_void_p]),
    "pstd_nn_gemm": (c_int, [c_void_p, c_void_p]),
    "pstd_nn_gemm_tf32": (c_int, [c_void_p, c_void_p, c_void_p]),
    "pstd_nn_bias_act": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int64, c_int, c_void_p]),
    "pstd_nn_act_bwd": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_void_p]),
    "pstd_nn_lift": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int64, c_void_p]),
    "pstd_nn_proj": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int64, c_void_p]),
    "pstd_nn_proj_bwd": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int64, c_void_p]),
    "pstd_nn_chan_dot": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int64, c_int, c_int64, c_void_p]),
    "pstd_nn_sum_lead": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "pstd_nn_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_float, c_float,
                             c_float, c_int64, c_void_p]),
    "pstd_nn_mse": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "pstd_nn_rel_err": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "pstd_nn_round_bf16": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "pstd_nn_row_rms": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "pstd_nn_row_scale": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p]),
    "pstd_sno_basis": (c_int, [c_int, c_int, c_int, c_int, POINTER(c_float), POINTER(c_float)]),
}


class PstdDesc(ctypes.Structure):
    """Mirror of pstd_desc."""
    _fields_ = [
        ("ndim", c_int),
        ("ncells", c_int64 * 3),
        ("dx", c_double * 3),
        ("bc", (c_int * 2) * 3),
        ("c0", c_double),
        ("rho0", c_double),
        ("dt", c_double),
        ("uinit", c_int),
    ]


class PstdGemmDesc(ctypes.Structure):
    """Mirror of pstd_gemm_desc."""
    _fields_ = [("batch", c_int64), ("M", c_int), ("N", c_int), ("K", c_int),
                ("A", c_void_p), ("sAb", c_int64), ("sAm", c_int64), ("sAk", c_int64),
                ("B", c_void_p), ("sBb", c_int64), ("sBk", c_int64), ("sBn", c_int64),
                ("C", c_void_p), ("sCb", c_int64), ("sCm", c_int64), ("sCn", c_int64),
                ("alpha", c_float), ("beta", c_float),
                ("batch2", c_int64), ("sAb2", c_int64), ("sBb2", c_int64), ("sCb2", c_int64), ("K_last", c_int)]


class PstdPlanOpts(ctypes.Structure):
    """Mirror of pstd_plan_opts (-1 = automatic)."""
    _fields_ = [("variant", c_int * 3), ("seqs_per_cta", c_int * 3), ("form", c_int),
                ("persistent", c_int), ("spin_limit", c_int64), ("withhold_arrivals", c_int)]


class PstdError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        msg = f"{what}: {ERRORS.get(code, code)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_LIBS = {}


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libpstd.so and declare its symbols; raises if it is not built."""
    path = path or LIB_PATH
    if path in _LIBS:
        return _LIBS[path]
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -m paper_2005_00322_gb300.build or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIBS[path] = lib
    return lib


def check(lib, code: int, what: str) -> None:
    if code != 0:
        detail = ""
        if code == -4:
            detail = (lib.pstd_last_cuda_error() or b"").decode()
        raise PstdError(code, what, detail)


def make_desc(ncells, dx, bc, c0, rho0, dt, uinit=U_HALFSTEP) -> PstdDesc:
    """Build a pstd_desc; bc per axis is a pair of "N" / "D" / "P" (right wall
    also "Nm" / "Dm": at mid-cell), or their codes."""
    d = PstdDesc()
    d.ndim = len(ncells)
    dxs = list(dx) if hasattr(dx, "__len__") else [dx]
    if len(dxs) == 1:
        dxs = dxs * d.ndim
    for i in range(3):
        d.ncells[i] = int(ncells[i]) if i < d.ndim else 1
        d.dx[i] = float(dxs[i]) if i < d.ndim else 1.0
        for s in range(2):
            if i < d.ndim:
                b = bc[i][s]
                d.bc[i][s] = BC_CODES.get(b, b) if isinstance(b, str) else int(b)
            else:
                d.bc[i][s] = NEUMANN
    d.c0, d.rho0, d.dt, d.uinit = float(c0), float(rho0), float(dt), int(uinit)
    return d
