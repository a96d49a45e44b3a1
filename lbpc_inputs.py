"""Seeded synthetic inputs and workload presets shared by the oracle and the CUDA path.

This module holds plain data only: the physical parameter block, the named
workloads shaped like the paper's test cases (Sec. 3.1.1 Stefan melting,
Sec. 3.1.2 solidification, Sec. 3.3 cubic-cavity melting) and seeded random
arrays.  It contains none of the method's arithmetic; the lattice mapping, the
equilibria and the collision live separately in ``oracle/`` and in the CUDA
library.

Random numbers (the enthalpy perturbation, the wall temperature field, random
test states) are drawn here once, on the host with ``numpy.random.default_rng``,
and the same arrays are handed to both implementations.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

# boundary codes of the six faces (-x, +x, -y, +y, -z, +z)
PERIODIC, ISOTHERMAL, ADIABATIC = 0, 1, 2
FLOW_NONE, FLOW_MRT, FLOW_SRT = 0, 1, 2
ENTH_MRT, ENTH_SRT = 1, 2
FP64, FP32, FP16, BF16, FP16_G32, BF16_G32 = 0, 1, 2, 3, 4, 5
PULL, AA = 0, 1
PRECISION_NAMES = {FP64: "f64", FP32: "f32", FP16: "f16s", BF16: "bf16s", FP16_G32: "f16s-g32",
                   BF16_G32: "bf16s-g32"}


@dataclass
class Params:
    """Physical inputs of one run (mirrors the C parameter block field by field)."""

    flow_model: int = FLOW_MRT
    enth_model: int = ENTH_MRT
    precision: int = FP32
    streaming: int = PULL
    bc: list = field(default_factory=lambda: [ISOTHERMAL, ISOTHERMAL, ADIABATIC, ADIABATIC,
                                              ADIABATIC, ADIABATIC])
    T_wall: list = field(default_factory=lambda: [1.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    Ra: float = 1e5
    Pr: float = 0.02
    St: float = 1.0
    Ma: float = 0.1
    Th: float = 1.0
    Tm: float = 0.0
    Tref: float = 0.5
    Cp_s: float = 1.0
    Cp_l: float = 1.0
    Cp_ref: float = 1.0
    omega_T: float = 0.25
    tau_g: float = 0.0
    nu: float = 0.0
    s_e: float = 0.0
    s_eps: float = 0.0
    s_q: float = 0.0
    s_pi: float = 0.0
    s_t: float = 0.0
    sigma4: float = 0.0
    h0: float = 0.0
    report_every: int = 0
    lambda_s: float = 0.0  # both > 0: per-phase conductivities (conduction only)
    lambda_l: float = 0.0
    darcy_A: float = 0.0  # > 0: enthalpy-porosity solid drag instead of the f_l closure
    darcy_eps: float = 0.0  # <= 0: 1e-3

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, bc=list(self.bc), T_wall=list(self.T_wall), **kw)


@dataclass
class Workload:
    name: str
    shape: tuple  # (nx, ny, nz)
    params: Params
    steps: int
    seed: int = 0
    perturb: float = 0.0  # amplitude of the uniform initial enthalpy perturbation

    @property
    def nodes(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def stefan_melting(nx=64, ny=4, nz=4, enth_model=ENTH_MRT, precision=FP64, streaming=PULL,
                   tau_g=0.8, St=0.1, sigma4=0.0) -> Workload:
    """1D melting of a half-space initially at T_m (Sec. 3.1.1): hot isothermal wall
    at x = -1/2 (T = 1), adiabatic far wall, periodic y and z, conduction only."""
    p = Params(flow_model=FLOW_NONE, enth_model=enth_model, precision=precision,
               streaming=streaming, bc=[ISOTHERMAL, ADIABATIC, PERIODIC, PERIODIC, PERIODIC,
                                        PERIODIC],
               T_wall=[1.0, 0.0, 0.0, 0.0, 0.0, 0.0], St=St, tau_g=tau_g, h0=0.0,
               sigma4=sigma4)
    return Workload(f"stefan-melting-{nx}x{ny}x{nz}", (nx, ny, nz), p, 5000)


def stefan_solidification(nx=64, ny=2, nz=2, chi=0.4, Ste=0.004, precision=FP64) -> Workload:
    """1D solidification of a half-space initially liquid at T_0 = 1 with the wall held
    at T_1 = -1 (Sec. 3.1.2 case (a): C_p,s = C_p,l = 1, Ste_s = Ste_l, equal
    diffusivities).  The Stefan number enters through St = C_p (T_m - T_1) / L."""
    omega_T = 0.25
    tau_g = chi / omega_T + 0.5
    # Th - Tm is the temperature scale of St; here the scale is T_m - T_1 = 1.
    L = 1.0 / Ste
    p = Params(flow_model=FLOW_NONE, enth_model=ENTH_MRT, precision=precision,
               bc=[ISOTHERMAL, ADIABATIC, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
               T_wall=[-1.0, 0.0, 0.0, 0.0, 0.0, 0.0], St=Ste, Th=1.0, Tm=0.0,
               tau_g=tau_g, omega_T=omega_T, h0=L + 1.0)
    return Workload(f"stefan-solidification-{nx}", (nx, ny, nz), p, 4000)


def stefan_solidification_b(nx=128, ny=2, nz=2, lambda_s=0.24, precision=FP64) -> Workload:
    """Sec. 3.1.2 case (b): C_p,s = 1, C_p,l = 2, Ste_s = 0.004, Ste_l = 0.008 and
    lambda_s / lambda_l = 0.6 / 0.15, so chi_s / chi_l = 8 (lattice units: lambda_s given,
    rho0 = C_p,ref = 1).  Initially liquid at T_0 = 1, wall at T_1 = -1, T_m = 0:
    L = C_p,l (T_0 - T_m) / Ste_l = 250, i.e. St = Ste_l with Th = T_0."""
    lambda_l = lambda_s * 0.15 / 0.6
    Cp_s, Cp_l = 1.0, 2.0
    L = Cp_l * 1.0 / 0.008
    p = Params(flow_model=FLOW_NONE, enth_model=ENTH_MRT, precision=precision,
               bc=[ISOTHERMAL, ADIABATIC, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
               T_wall=[-1.0, 0.0, 0.0, 0.0, 0.0, 0.0], St=0.008, Th=1.0, Tm=0.0,
               Cp_s=Cp_s, Cp_l=Cp_l, Cp_ref=1.0, omega_T=0.25,
               lambda_s=lambda_s, lambda_l=lambda_l, h0=L + Cp_l * 1.0)
    return Workload(f"stefan-solidification-b-{nx}", (nx, ny, nz), p, 20000)


def cavity_melting(n=64, Ra=1e5, Pr=0.02, St=1.0, precision=FP32, streaming=PULL,
                   flow_model=FLOW_MRT, enth_model=ENTH_MRT, steps=20000, report_every=500,
                   shape=None) -> Workload:
    """Cubic-cavity melting (Sec. 3.3): hot isothermal wall x = -1/2 at T = 1, cold
    wall x = n - 1/2 at T = T_m = 0, other faces adiabatic; all faces no-slip;
    initially solid at T_m with a seeded uniform +-1e-6 enthalpy perturbation."""
    p = Params(flow_model=flow_model, enth_model=enth_model, precision=precision,
               streaming=streaming, Ra=Ra, Pr=Pr, St=St, report_every=report_every)
    shape = tuple(shape) if shape is not None else (n, n, n)
    name = f"cavity-melting-{shape[0]}x{shape[1]}x{shape[2]}-Ra{Ra:g}-Pr{Pr:g}-St{St:g}"
    return Workload(name, shape, p, steps, seed=0, perturb=1e-6)


def corner_solidification(n=128, chi=0.1, precision=FP64) -> Workload:
    """2D solidification in a corner (Sec. 3.2.1): liquid at T_0 = 0.3 in x, z > 0, the
    planes x = -1/2 and z = -1/2 held at T_1 = -1 from t = 0, T_f = 0; equal properties,
    Ste_s = C_p (T_f - T_1) / L = 4 (L = 1/4, so St = C_p (T_0 - T_f) / L = 1.2); one
    periodic node along y, adiabatic far faces; conduction only with chi given."""
    L = 0.25
    p = Params(flow_model=FLOW_NONE, enth_model=ENTH_MRT, precision=precision,
               bc=[ISOTHERMAL, ADIABATIC, PERIODIC, PERIODIC, ISOTHERMAL, ADIABATIC],
               T_wall=[-1.0, 0.0, 0.0, 0.0, -1.0, 0.0], St=0.3 / L, Th=0.3, Tm=0.0,
               tau_g=chi / 0.25 + 0.5, h0=L + 0.3)
    return Workload(f"corner-solidification-{n}x1x{n}", (n, 1, n), p, 4500)


def cavity_melting_2d(n=64, Ra=2.5e4, Pr=0.02, St=0.01, precision=FP32, steps=100000,
                      report_every=0) -> Workload:
    """Quasi-2D convective melting (Sec. 3.2.2, Table 1): a 1 x 1 cavity in x-z, infinite
    along y (one periodic node); hot wall x = -1/2 at T = 1, cold wall x = n - 1/2 at
    T = T_m = 0, top and bottom (z) adiabatic, all walls no-slip; gravity along -z;
    initially solid at T_m with a seeded +-1e-6 enthalpy perturbation."""
    p = Params(flow_model=FLOW_MRT, enth_model=ENTH_MRT, precision=precision,
               bc=[ISOTHERMAL, ISOTHERMAL, PERIODIC, PERIODIC, ADIABATIC, ADIABATIC],
               T_wall=[1.0, 0.0, 0.0, 0.0, 0.0, 0.0], Ra=Ra, Pr=Pr, St=St,
               report_every=report_every)
    return Workload(f"cavity-melting-2d-{n}x1x{n}-Ra{Ra:g}-Pr{Pr:g}-St{St:g}", (n, 1, n), p,
                    steps, seed=0, perturb=1e-6)


def h0_field(w: Workload) -> np.ndarray:
    """Initial enthalpy per node: the uniform h0 plus the seeded perturbation."""
    h = np.full(w.nodes, w.params.h0, dtype=np.float64)
    if w.perturb > 0:
        rng = np.random.default_rng(w.seed)
        h += rng.uniform(-w.perturb, w.perturb, size=w.nodes)
    return h


def wall_temperature_field(ny: int, nz: int, seed: int = 0, mean=1.0, std=0.05) -> np.ndarray:
    """Per-node hot-wall temperature T_w(y, z) = 1 + 0.05 N(0, 1), seeded; y fastest."""
    rng = np.random.default_rng(seed)
    return mean + std * rng.standard_normal(ny * nz)


def fd_wall_nodes(ny: int, nz: int, count: int = 16, seed: int = 0) -> np.ndarray:
    """Seeded distinct wall nodes (flat index y + ny z) for finite-difference checks."""
    rng = np.random.default_rng(seed + 1)
    return np.sort(rng.choice(ny * nz, size=count, replace=False))


def random_state(shape, seed: int = 0, h_range=(-0.5, 2.5), flow=True):
    """A seeded random pre-collision state: f (19, N) and g (7, N) in float64.

    f_a is positive with sum near 1; g_1..6 are positive, g_0 takes the rest of a
    random enthalpy drawn across solid, mushy and liquid values.  Used to drive
    one-step comparisons from a state far from equilibrium."""
    nx, ny, nz = shape
    N = nx * ny * nz
    rng = np.random.default_rng(seed)
    f = None
    if flow:
        f = (1.0 / 19.0) * (1.0 + 0.3 * rng.uniform(-1.0, 1.0, size=(19, N)))
    h = rng.uniform(h_range[0], h_range[1], size=N)
    g = np.empty((7, N))
    g[1:] = rng.uniform(0.0, 0.25, size=(6, N))
    g[0] = h - g[1:].sum(axis=0)
    return f, g


def bench_workload() -> Workload:
    """The timed workload: 256^3 cavity melting, Ra = 1e6, Pr = 0.02, St = 1, D3Q19 MRT
    flow + D3Q7 MRT enthalpy, FP32 storage, two-lattice pull streaming."""
    return cavity_melting(n=256, Ra=1e6, Pr=0.02, St=1.0, precision=FP32, streaming=PULL,
                          steps=50000, report_every=500)
