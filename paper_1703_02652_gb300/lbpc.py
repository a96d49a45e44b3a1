"""``LBPC``: one lattice on one GPU, driven through the C ABI.

PyTorch supplies the device workspace (a ``uint8`` tensor the handle carves its
populations out of) and the CUDA stream; every computation runs in ``liblbpc.so``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import binding as B


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _hptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


class LBPC:
    """Coupled D3Q19 flow + D3Q7 enthalpy lattice of shape (nx, ny, nz).

    ``params`` is an ``lbpc_inputs.Params``.  The workspace lives on ``device``
    (default: the current CUDA device) and all work is queued on ``stream``
    (default: torch's current stream of that device)."""

    def __init__(self, shape, params, device=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("LBPC needs a CUDA device; there is no CPU implementation")
        self.shape = tuple(int(v) for v in shape)
        self.nx, self.ny, self.nz = self.shape
        self.N = self.nx * self.ny * self.nz
        self.params = params
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        L = B.lib()
        self._cp = B.to_c(params)
        nbytes = int(L.lbpc_workspace_bytes(self.nx, self.ny, self.nz, C.byref(self._cp)))
        if nbytes == 0:
            # surfaces the validation message
            h = C.c_void_p()
            st = L.lbpc_create(self.nx, self.ny, self.nz, C.byref(self._cp), None, 0, None,
                               C.byref(h))
            B.check(st, None)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = C.c_void_p()
        st = L.lbpc_create(self.nx, self.ny, self.nz, C.byref(self._cp),
                           C.c_void_p(self.workspace.data_ptr()), nbytes,
                           C.c_void_p(self.stream.cuda_stream), C.byref(self._h))
        B.check(st, None)
        self.flow = params.flow_model != 0

    # ------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            B.lib().lbpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        B.check(st, self._h)

    # -- set-up ----------------------------------------------------------------------
    def set_initial_h(self, h):
        h = np.ascontiguousarray(h, dtype=np.float64).reshape(-1)
        assert h.size == self.N
        self._check(B.lib().lbpc_set_initial_h(self._h, _hptr(h)))

    def set_wall_temperature(self, face: int, T):
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        self._check(B.lib().lbpc_set_wall_temperature(self._h, int(face), _hptr(T)))

    # -- time stepping ---------------------------------------------------------------
    def step(self, n: int = 1):
        self._check(B.lib().lbpc_step(self._h, int(n)))

    @property
    def step_count(self) -> int:
        return int(B.lib().lbpc_step_count(self._h))

    @property
    def launch_count(self) -> int:
        """Kernels this handle has launched since creation."""
        return int(B.lib().lbpc_launch_count(self._h))

    # -- read-out --------------------------------------------------------------------
    def fields(self):
        """FP64 device tensors T, fl, h, rho (nz, ny, nx) and u (3, nz, ny, nx)."""
        kw = dict(dtype=torch.float64, device=self.device)
        T = torch.empty(self.N, **kw); fl = torch.empty(self.N, **kw)
        h = torch.empty(self.N, **kw); rho = torch.empty(self.N, **kw)
        u = torch.empty(3 * self.N, **kw)
        self._check(B.lib().lbpc_get_fields_dev(self._h, _dptr(T), _dptr(fl), _dptr(h),
                                                _dptr(rho), _dptr(u)))
        sh = (self.nz, self.ny, self.nx)
        return {"T": T.view(sh), "fl": fl.view(sh), "h": h.view(sh), "rho": rho.view(sh),
                "u": u.view((3,) + sh)}

    def fields_host(self, mask=B.FIELD_T | B.FIELD_FL | B.FIELD_H | B.FIELD_RHO | B.FIELD_U):
        """Same fields copied to host numpy arrays through the host-pointer entry point."""
        out = {k: np.empty(self.N) for k in ("T", "fl", "h", "rho")}
        u = np.empty(3 * self.N)
        self._check(B.lib().lbpc_get_fields(self._h, int(mask), _hptr(out["T"]),
                                            _hptr(out["fl"]), _hptr(out["h"]),
                                            _hptr(out["rho"]), _hptr(u)))
        sh = (self.nz, self.ny, self.nx)
        res = {k: v.reshape(sh) for k, v in out.items()}
        res["u"] = u.reshape((3,) + sh)
        return res

    def scalars(self) -> dict:
        out = np.zeros(len(B.S_NAMES))
        self._check(B.lib().lbpc_get_scalars(self._h, _hptr(out), out.size))
        return dict(zip(B.S_NAMES, out.tolist()))

    def history(self) -> np.ndarray:
        out = np.zeros((B.HISTORY_ROWS, len(B.S_NAMES)))
        rows = C.c_int(0)
        self._check(B.lib().lbpc_get_history(self._h, _hptr(out), B.HISTORY_ROWS, C.byref(rows)))
        return out[: rows.value]

    def lattice(self) -> dict:
        out = np.zeros(len(B.L_NAMES))
        self._check(B.lib().lbpc_get_lattice(self._h, _hptr(out), out.size))
        return dict(zip(B.L_NAMES, out.tolist()))

    def distributions(self):
        """Pre-collision populations (FP64 device tensors): f (19, N) or None, g (7, N)."""
        kw = dict(dtype=torch.float64, device=self.device)
        g = torch.empty((7, self.N), **kw)
        f = torch.empty((19, self.N), **kw) if self.flow else None
        self._check(B.lib().lbpc_get_distributions_dev(self._h, _dptr(f), _dptr(g)))
        return f, g

    def set_distributions(self, f, g):
        """Load a pre-collision state from FP64 device tensors f (19, N) and g (7, N)."""
        g = g.to(self.device, torch.float64).contiguous()
        if f is not None:
            f = f.to(self.device, torch.float64).contiguous()
        self._check(B.lib().lbpc_set_distributions_dev(self._h, _dptr(f if self.flow else None),
                                                       _dptr(g)))
        self.stream.synchronize()

    # -- adjoint ---------------------------------------------------------------------
    def _face_area(self, face):
        return [self.ny * self.nz] * 2 + [self.nx * self.nz] * 2 + [self.nx * self.ny] * 2

    def adjoint_forward(self, nsteps: int, ckpt_every: int) -> float:
        """Advance nsteps with checkpoints; returns J = sum f_l at the end.  The adjoint
        workspace (a torch uint8 tensor) is kept on the object for adjoint_backward."""
        n = int(B.lib().lbpc_adjoint_workspace_bytes(self._h, int(nsteps), int(ckpt_every)))
        if n == 0:
            raise ValueError("invalid nsteps / ckpt_every")
        ws = getattr(self, "_adj_ws", None)
        if ws is None or ws.numel() < n:
            self._adj_ws = None
            self._adj_ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        J = C.c_double()
        self._check(B.lib().lbpc_adjoint_forward(self._h, int(nsteps), int(ckpt_every),
                                                 C.c_void_p(self._adj_ws.data_ptr()),
                                                 self._adj_ws.numel(), C.byref(J)))
        return J.value

    def adjoint_backward(self, face: int = 0):
        """Gradients of the last adjoint_forward's J: (dJ/dT_w of `face`, dJ/dSt)."""
        g = np.zeros(self._face_area(face)[face])
        dSt = C.c_double()
        self._check(B.lib().lbpc_adjoint_backward(self._h, int(face), _hptr(g), C.byref(dSt)))
        return g, dSt.value

    def adjoint(self, nsteps: int, ckpt_every: int, face: int = 0):
        """(J, dJ/dT_w of `face`, dJ/dSt) for nsteps steps from the current state."""
        J = self.adjoint_forward(nsteps, ckpt_every)
        g, dSt = self.adjoint_backward(face)
        return J, g, dSt

    def release_adjoint_workspace(self):
        self._adj_ws = None

    # -- checkpoint ------------------------------------------------------------------
    def save(self) -> bytes:
        n = int(B.lib().lbpc_state_bytes(self._h))
        buf = C.create_string_buffer(n)
        self._check(B.lib().lbpc_save(self._h, buf, n))
        return buf.raw

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(B.lib().lbpc_load(self._h, buf, len(blob)))
