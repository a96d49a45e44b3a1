"""ctypes binding of ``liblbpc.so`` (the C ABI of ``include/lbpc.h``).

Argument marshalling only: every step of the method runs in the CUDA library.  The
library is built in-tree (``_build.build()``); importing this module without it
raises, there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

LBPC_OK, LBPC_ERR_PARAM, LBPC_ERR_WORKSPACE, LBPC_ERR_CUDA, LBPC_ERR_DIVERGED, LBPC_ERR_STATE = (
    0, -1, -2, -3, -4, -5)
STATUS_NAMES = {0: "OK", -1: "ERR_PARAM", -2: "ERR_WORKSPACE", -3: "ERR_CUDA", -4: "ERR_DIVERGED",
                -5: "ERR_STATE"}
FIELD_T, FIELD_FL, FIELD_H, FIELD_RHO, FIELD_U = 1, 2, 4, 8, 16
S_NAMES = ["liquid_vol", "nu_hot", "front_mean", "sum_h", "sum_rho", "step", "nu_fd",
           "front_mid", "nan"]
L_NAMES = ["chi", "nu", "gbeta", "sigma_chi", "sigma4", "s_nu", "latent", "hs", "hl", "tau_g",
           "tau_f", "s_e", "s_eps", "s_q", "s_pi", "s_t", "U0"]
HISTORY_ROWS = 4096

# every symbol include/lbpc.h declares
EXPORTS = ["lbpc_params_size", "lbpc_abi_version", "lbpc_workspace_bytes", "lbpc_create",
           "lbpc_set_initial_h", "lbpc_set_wall_temperature", "lbpc_step", "lbpc_get_fields",
           "lbpc_get_fields_dev", "lbpc_get_scalars", "lbpc_get_history",
           "lbpc_get_distributions_dev", "lbpc_set_distributions_dev", "lbpc_get_lattice",
           "lbpc_lattice_constants", "lbpc_adjoint_workspace_bytes", "lbpc_adjoint_forward",
           "lbpc_adjoint_backward", "lbpc_adjoint", "lbpc_get_scalars_noalloc",
           "lbpc_state_bytes", "lbpc_save", "lbpc_load", "lbpc_step_count", "lbpc_launch_count",
           "lbpc_last_error",
           "lbpc_destroy"]


class LbpcParams(C.Structure):
    _fields_ = [("flow_model", C.c_int), ("enth_model", C.c_int), ("precision", C.c_int),
                ("streaming", C.c_int), ("bc", C.c_int * 6), ("T_wall", C.c_double * 6)] + [
        (n, C.c_double) for n in ("Ra", "Pr", "St", "Ma", "Th", "Tm", "Tref", "Cp_s", "Cp_l",
                                  "Cp_ref", "omega_T", "tau_g", "nu", "s_e", "s_eps", "s_q",
                                  "s_pi", "s_t", "sigma4", "h0")] + [("report_every", C.c_int)] + [
        ("lambda_s", C.c_double), ("lambda_l", C.c_double), ("darcy_A", C.c_double),
        ("darcy_eps", C.c_double)]


class LbpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib(build: bool = True):
    """Load liblbpc.so (building it first when sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, d, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
    L.lbpc_params_size.restype = sz
    L.lbpc_abi_version.restype = C.c_int
    L.lbpc_workspace_bytes.restype = sz
    L.lbpc_workspace_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(LbpcParams)]
    L.lbpc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(LbpcParams), vp, sz, vp,
                              C.POINTER(vp)]
    L.lbpc_set_initial_h.argtypes = [vp, d]
    L.lbpc_set_wall_temperature.argtypes = [vp, C.c_int, d]
    L.lbpc_step.argtypes = [vp, C.c_int]
    L.lbpc_get_fields.argtypes = [vp, C.c_uint, d, d, d, d, d]
    L.lbpc_get_fields_dev.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lbpc_get_scalars.argtypes = [vp, d, C.c_int]
    L.lbpc_get_history.argtypes = [vp, d, C.c_int, C.POINTER(C.c_int)]
    L.lbpc_get_distributions_dev.argtypes = [vp, vp, vp]
    L.lbpc_set_distributions_dev.argtypes = [vp, vp, vp]
    L.lbpc_get_lattice.argtypes = [vp, d, C.c_int]
    L.lbpc_lattice_constants.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(LbpcParams), d,
                                         C.c_int]
    L.lbpc_adjoint_workspace_bytes.restype = sz
    L.lbpc_adjoint_workspace_bytes.argtypes = [vp, C.c_int, C.c_int]
    L.lbpc_adjoint_forward.argtypes = [vp, C.c_int, C.c_int, vp, sz, d]
    L.lbpc_adjoint_backward.argtypes = [vp, C.c_int, d, d]
    L.lbpc_adjoint.argtypes = [vp, C.c_int, C.c_int, vp, sz, C.c_int, d, d, d]
    L.lbpc_get_scalars_noalloc.argtypes = [vp, vp]
    L.lbpc_state_bytes.restype = sz
    L.lbpc_state_bytes.argtypes = [vp]
    L.lbpc_save.argtypes = [vp, vp, sz]
    L.lbpc_load.argtypes = [vp, vp, sz]
    L.lbpc_step_count.restype = C.c_longlong
    L.lbpc_step_count.argtypes = [vp]
    L.lbpc_launch_count.restype = C.c_longlong
    L.lbpc_launch_count.argtypes = [vp]
    L.lbpc_last_error.restype = C.c_char_p
    L.lbpc_last_error.argtypes = [vp]
    L.lbpc_destroy.argtypes = [vp]
    L.lbpc_destroy.restype = None
    _lib = L
    return L


def to_c(params) -> LbpcParams:
    """Copy a ``lbpc_inputs.Params`` (or any object with the same fields) into the C block."""
    cp = LbpcParams()
    for name, _ in LbpcParams._fields_:
        v = getattr(params, name)
        if name in ("bc", "T_wall"):
            arr = getattr(cp, name)
            for i in range(6):
                arr[i] = v[i]
        else:
            setattr(cp, name, v)
    return cp


def check(status: int, handle=None):
    if status != LBPC_OK:
        msg = lib().lbpc_last_error(handle)
        raise LbpcError(status, msg.decode() if msg else "")


def workspace_bytes(shape, params) -> int:
    cp = to_c(params)
    return int(lib().lbpc_workspace_bytes(shape[0], shape[1], shape[2], C.byref(cp)))


def lattice_constants(shape, params) -> dict:
    """Derived lattice constants of a parameter block (host only, no device needed)."""
    import numpy as np
    cp = to_c(params)
    out = np.zeros(len(L_NAMES))
    st = lib().lbpc_lattice_constants(shape[0], shape[1], shape[2], C.byref(cp),
                                      out.ctypes.data_as(C.POINTER(C.c_double)), out.size)
    check(st, None)
    return dict(zip(L_NAMES, out.tolist()))
