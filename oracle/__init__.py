"""FP64 CPU oracle of the coupled enthalpy / flow lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it.

``liblbpc_oracle.so`` is built from ``lbpc_oracle.c`` with gcc (OpenMP when
available).  This module is argument marshalling only: every step of the method
runs in the C file, which cites the paper's equations line by line.

Parity pins of this oracle: see ``tests/test_oracle_pins.py`` and
``tests/test_oracle_analytic.py``.  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbpc_oracle.c")
_SRC_ADJ = os.path.join(_HERE, "lbpc_oracle_adjoint.c")
_LIB = os.path.join(_HERE, "liblbpc_oracle.so")

L_NAMES = ["chi", "nu", "gbeta", "sigma_chi", "sigma4", "s_nu", "latent", "hs", "hl", "tau_g",
           "tau_f", "s_e", "s_eps", "s_q", "s_pi", "s_t", "U0"]
D_NAMES = ["liquid_vol", "nu_hot", "front_mean", "sum_h", "sum_rho", "step", "nu_fd",
           "front_mid", "nan"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the path of the shared library."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_ADJ),
            os.path.getmtime(os.path.join(_HERE, "lbpc_oracle.h"))):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", _LIB + ".tmp", _SRC,
            _SRC_ADJ, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("flow_model", C.c_int), ("enth_model", C.c_int), ("bc", C.c_int * 6),
                ("T_wall", C.c_double * 6)] + [
        (n, C.c_double) for n in ("Ra", "Pr", "St", "Ma", "Th", "Tm", "Tref", "Cp_s", "Cp_l",
                                  "Cp_ref", "omega_T", "tau_g", "nu", "s_e", "s_eps", "s_q",
                                  "s_pi", "s_t", "sigma4", "h0", "lambda_s", "lambda_l",
                                  "darcy_A", "darcy_eps")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        _lib.orc_create.restype = C.c_void_p
        _lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(_Params), C.c_int]
        _lib.orc_destroy.argtypes = [C.c_void_p]
        _lib.orc_last_error.restype = C.c_char_p
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_threads.restype = C.c_int
        _lib.orc_set_initial_h.argtypes = [C.c_void_p, d]
        _lib.orc_set_wall_temperature.argtypes = [C.c_void_p, C.c_int, d]
        _lib.orc_set_distributions.argtypes = [C.c_void_p, d, d]
        _lib.orc_step.argtypes = [C.c_void_p, C.c_int]
        _lib.orc_fields.argtypes = [C.c_void_p, d, d, d, d, d]
        _lib.orc_distributions.argtypes = [C.c_void_p, d, d]
        _lib.orc_diagnostics.argtypes = [C.c_void_p, d]
        _lib.orc_lattice.argtypes = [C.c_void_p, d]
        _lib.orc_wall_flux.argtypes = [C.c_void_p, C.c_int, d]
        _lib.orc_step_count.restype = C.c_long
        _lib.orc_step_count.argtypes = [C.c_void_p]
        _lib.orc_update_sampled.argtypes = [C.c_void_p, d, d, C.c_long,
                                            C.POINTER(C.c_long), d, d]
        _lib.orc_tables.argtypes = [d, d, d, d, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _lib.orc_invert.argtypes = [C.c_void_p, C.c_double, d, d]
        _lib.orc_flow_meq.argtypes = [C.c_double, d, d]
        _lib.orc_flow_forcing.argtypes = [d, d, d]
        _lib.orc_enth_geq.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, d, d]
        _lib.orc_enth_neq.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, d, d]
        _lib.orc_collide_node.argtypes = [C.c_void_p, d, d, d, d, d]
        _lib.orc_adjoint.argtypes = [C.c_void_p, C.c_int, C.c_int, d, d, d]
        _lib.orc_collide_jacobian.argtypes = [C.c_void_p, d, d, d, d]
    return _lib


def _p(a):
    """Pointer to a C-contiguous float64 array (None -> NULL)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _to_c(params) -> _Params:
    cp = _Params()
    cp.flow_model = params.flow_model
    cp.enth_model = params.enth_model
    for i in range(6):
        cp.bc[i] = int(params.bc[i])
        cp.T_wall[i] = float(params.T_wall[i])
    for n, _ in _Params._fields_[4:]:
        setattr(cp, n, float(getattr(params, n)))
    return cp


def tables():
    """(M, Minv, N, Ninv, e19, e7) as the oracle holds them."""
    M = np.zeros(361); Mi = np.zeros(361); N = np.zeros(49); Ni = np.zeros(49)
    e19 = (C.c_int * 57)(); e7 = (C.c_int * 21)()
    lib().orc_tables(_p(M), _p(Mi), _p(N), _p(Ni), e19, e7)
    return (M.reshape(19, 19), Mi.reshape(19, 19), N.reshape(7, 7), Ni.reshape(7, 7),
            np.array(e19[:]).reshape(19, 3), np.array(e7[:]).reshape(7, 3))


def flow_meq(rho, u):
    out = np.zeros(19)
    lib().orc_flow_meq(float(rho), _p(np.asarray(u, dtype=np.float64).copy()), _p(out))
    return out


def flow_forcing(F, u):
    out = np.zeros(19)
    lib().orc_flow_forcing(_p(np.asarray(F, dtype=np.float64).copy()),
                           _p(np.asarray(u, dtype=np.float64).copy()), _p(out))
    return out


def set_threads(n: int):
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_threads())


class Oracle:
    """One oracle lattice; holds the pre-collision state at the current time."""

    def __init__(self, shape, params, alloc: bool = True):
        self.shape = tuple(int(v) for v in shape)
        self.nx, self.ny, self.nz = self.shape
        self.N = self.nx * self.ny * self.nz
        self.params = params
        self._cp = _to_c(params)
        self._h = lib().orc_create(self.nx, self.ny, self.nz, C.byref(self._cp), int(alloc))
        if not self._h:
            raise ValueError("oracle: " + lib().orc_last_error().decode())
        self.flow = params.flow_model != 0

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -----------------------------------------------------------------------
    def set_initial_h(self, h):
        h = np.ascontiguousarray(h, dtype=np.float64)
        assert h.size == self.N
        if lib().orc_set_initial_h(self._h, _p(h)) != 0:
            raise RuntimeError(lib().orc_last_error().decode())

    def set_wall_temperature(self, face, T):
        T = np.ascontiguousarray(T, dtype=np.float64)
        if lib().orc_set_wall_temperature(self._h, int(face), _p(T)) != 0:
            raise RuntimeError(lib().orc_last_error().decode())

    def set_distributions(self, f, g):
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(7, self.N)
        fp = None
        if f is not None and self.flow:
            f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
            fp = _p(f)
        if lib().orc_set_distributions(self._h, fp, _p(g)) != 0:
            raise RuntimeError(lib().orc_last_error().decode())

    # -- stepping and read-out --------------------------------------------------------
    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return int(lib().orc_step_count(self._h))

    def fields(self):
        """dict of FP64 fields over the lattice, each shaped (nz, ny, nx); u is (3, nz, ny, nx)."""
        T = np.empty(self.N); fl = np.empty(self.N); h = np.empty(self.N)
        rho = np.empty(self.N); u = np.empty(3 * self.N)
        lib().orc_fields(self._h, _p(T), _p(fl), _p(h), _p(rho), _p(u))
        sh = (self.nz, self.ny, self.nx)
        return {"T": T.reshape(sh), "fl": fl.reshape(sh), "h": h.reshape(sh),
                "rho": rho.reshape(sh), "u": u.reshape((3,) + sh)}

    def distributions(self):
        f = np.zeros(19 * self.N); g = np.empty(7 * self.N)
        lib().orc_distributions(self._h, _p(f), _p(g))
        return f.reshape(19, self.N), g.reshape(7, self.N)

    def diagnostics(self) -> dict:
        out = np.zeros(len(D_NAMES))
        lib().orc_diagnostics(self._h, _p(out))
        return dict(zip(D_NAMES, out.tolist()))

    def lattice(self) -> dict:
        out = np.zeros(len(L_NAMES))
        lib().orc_lattice(self._h, _p(out))
        return dict(zip(L_NAMES, out.tolist()))

    def wall_flux(self, face: int):
        A = [self.ny * self.nz] * 2 + [self.nx * self.nz] * 2 + [self.nx * self.ny] * 2
        q = np.empty(A[face])
        lib().orc_wall_flux(self._h, int(face), _p(q))
        return q

    # -- node-level operations -------------------------------------------------------
    def invert(self, h):
        T = C.c_double(); fl = C.c_double()
        lib().orc_invert(self._h, float(h), C.byref(T), C.byref(fl))
        return T.value, fl.value

    def enth_geq(self, h, T, fl, u):
        out = np.zeros(7)
        lib().orc_enth_geq(self._h, float(h), float(T), float(fl),
                           _p(np.asarray(u, dtype=np.float64).copy()), _p(out))
        return out

    def enth_neq(self, h, T, fl, u):
        out = np.zeros(7)
        lib().orc_enth_neq(self._h, float(h), float(T), float(fl),
                           _p(np.asarray(u, dtype=np.float64).copy()), _p(out))
        return out

    def collide_node(self, f, g):
        """Post-collision (f*, g*) and macroscopics (h, T, fl, rho, u, F) of one node."""
        f = np.ascontiguousarray(f if f is not None else np.zeros(19), dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        fp = np.zeros(19); gp = np.zeros(7); mac = np.zeros(10)
        lib().orc_collide_node(self._h, _p(f), _p(g), _p(fp), _p(gp), _p(mac))
        return fp, gp, {"h": mac[0], "T": mac[1], "fl": mac[2], "rho": mac[3],
                        "u": mac[4:7].copy(), "F": mac[7:10].copy()}

    def collide_jacobian(self, f, g):
        """Exact Jacobian of the node collision (complex step) and its L-derivative."""
        n = 26 if self.flow else 7
        f = np.ascontiguousarray(f if f is not None else np.zeros(19), dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        J = np.zeros(n * n); dL = np.zeros(26)
        lib().orc_collide_jacobian(self._h, _p(f), _p(g), _p(J), _p(dL))
        return J.reshape(n, n), dL[:n]

    def adjoint(self, nsteps: int, face: int = 0):
        """Run nsteps forward; return J = sum f_l(h_N), dJ/dT_w(face) and dJ/dSt."""
        A = [self.ny * self.nz] * 2 + [self.nx * self.nz] * 2 + [self.nx * self.ny] * 2
        J = C.c_double(); dSt = C.c_double(); dTw = np.zeros(A[face])
        st = lib().orc_adjoint(self._h, int(nsteps), int(face), C.byref(J), _p(dTw), C.byref(dSt))
        if st != 0:
            raise RuntimeError("oracle adjoint failed")
        return J.value, dTw, dSt.value

    def update_sampled(self, f, g, idx):
        """New pre-collision populations of nodes ``idx`` after one step from (f, g)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        fptr = None
        if self.flow:
            f = np.ascontiguousarray(f, dtype=np.float64)
            fptr = _p(f)
        fo = np.zeros((idx.size, 19)); go = np.zeros((idx.size, 7))
        lib().orc_update_sampled(self._h, fptr, _p(g), idx.size,
                                 idx.ctypes.data_as(C.POINTER(C.c_long)), _p(fo), _p(go))
        return fo, go


def run(workload, steps=None, h0=None, wall=None, threads_=None):
    """Run a workload from its initial state; returns the Oracle object."""
    import lbpc_inputs as inp
    o = Oracle(workload.shape, workload.params)
    if threads_:
        set_threads(threads_)
    if wall is not None:
        for face, T in wall.items():
            o.set_wall_temperature(face, T)
    o.set_initial_h(h0 if h0 is not None else inp.h0_field(workload))
    o.step(workload.steps if steps is None else steps)
    return o


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
