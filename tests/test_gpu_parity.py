"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances, from the arithmetic of each storage mode:
* FP64 storage: the kernels evaluate the same equations as the oracle in another
  order (structured moment sums instead of dense 19x19 / 7x7 products), so results
  differ by accumulated FP64 rounding: 1e-11 absolute after tens of steps on O(1)
  fields; the 1D Stefan run (5000 steps) must meet the stated 1e-6 relative bound on T.
* FP32 storage / FP32 collision: one step from a state the oracle also starts from
  differs by FP32 rounding of moments up to ~30x the populations: 5e-6 absolute.
* FP16 / BF16 shifted storage: one rounding of the stored deviation per population per
  step; the random states reach deviations in [0.25, 0.5), where one ulp is 2.4e-4 (FP16)
  and 2.0e-3 (BF16).  The rest channel g_0 = h' absorbs the six roundings of g_1..6.
"""
import numpy as np
import pytest
import torch

import lbpc_inputs as inp
import oracle
from paper_1703_02652_gb300 import LBPC, LbpcError
from paper_1703_02652_gb300 import binding as B

pytestmark = pytest.mark.gpu

KEYS = ("T", "fl", "h", "rho", "u")


def _np(F):
    return {k: v.detach().cpu().numpy() for k, v in F.items()}


def _maxerr(A, R, keys=KEYS):
    return {k: float(np.abs(A[k] - R[k]).max()) for k in keys}


def _pair(shape, p, h0=None, walls=None):
    g = LBPC(shape, p)
    o = oracle.Oracle(shape, p)
    if walls:
        for face, T in walls.items():
            g.set_wall_temperature(face, T)
            o.set_wall_temperature(face, T)
    if h0 is not None:
        g.set_initial_h(h0)
        o.set_initial_h(h0)
    return g, o


# ------------------------------------------------------------------------------------
# 1D Stefan melting, 64x4x4, FP64 GPU mode: relative max error on T <= 1e-6
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("enth_model", [inp.ENTH_SRT, inp.ENTH_MRT])
@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
def test_stefan_melting_fp64(enth_model, streaming):
    w = inp.stefan_melting(enth_model=enth_model, streaming=streaming)
    g, o = _pair(w.shape, w.params, h0=inp.h0_field(w))
    g.step(w.steps)
    o.step(w.steps)
    A, R = _np(g.fields()), o.fields()
    rel_T = np.abs(A["T"] - R["T"]).max() / np.abs(R["T"]).max()
    assert rel_T <= 1e-6
    assert np.abs(A["fl"] - R["fl"]).max() <= 1e-9
    sg, so = g.scalars(), o.diagnostics()
    for k in ("liquid_vol", "front_mean", "nu_hot", "nu_fd", "front_mid", "sum_h"):
        assert abs(sg[k] - so[k]) <= 1e-9 * max(1.0, abs(so[k])), k
    assert sg["step"] == w.steps == o.step_count


# ------------------------------------------------------------------------------------
# 3D cavities with flow, FP64 storage, every model combination and both streamings
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("flow_model", [inp.FLOW_MRT, inp.FLOW_SRT])
@pytest.mark.parametrize("enth_model", [inp.ENTH_MRT, inp.ENTH_SRT])
@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
def test_cavity_fp64(flow_model, enth_model, streaming):
    shape = (13, 7, 9)
    p = inp.Params(flow_model=flow_model, enth_model=enth_model, precision=inp.FP64,
                   streaming=streaming, Ra=3e4, Pr=0.7, St=0.8)
    rng = np.random.default_rng(1)
    h0 = rng.uniform(-0.3, 2.0, int(np.prod(shape)))
    g, o = _pair(shape, p, h0=h0)
    g.step(61)  # odd: AA ends in its swapped layout
    o.step(61)
    err = _maxerr(_np(g.fields()), o.fields())
    assert max(err.values()) <= 1e-11, err
    assert np.abs(o.fields()["u"]).max() > 1e-4  # the flow was active


# the enthalpy-porosity solid drag in place of the liquid-fraction closure
@pytest.mark.parametrize("precision,streaming,tol", [
    (inp.FP64, inp.PULL, 1e-11), (inp.FP64, inp.AA, 1e-11), (inp.FP32, inp.PULL, 2e-4),
    (inp.FP32, inp.AA, 2e-4)])
def test_cavity_darcy_closure(precision, streaming, tol):
    shape = (14, 7, 9)  # even n_x: the paired kernels take the interior rows
    p = inp.Params(flow_model=inp.FLOW_MRT, precision=precision, streaming=streaming, Ra=3e4,
                   Pr=0.7, St=0.8, darcy_A=5.0)
    h0 = np.random.default_rng(1).uniform(-0.3, 2.0, int(np.prod(shape)))
    g, o = _pair(shape, p, h0=h0)
    g.step(61)
    o.step(61)
    err = _maxerr(_np(g.fields()), o.fields())
    assert max(err.values()) <= tol, err
    assert np.abs(o.fields()["u"]).max() > 1e-4


@pytest.mark.parametrize("darcy_A,fl0", [(0.0, 0.3), (1.0, 0.3), (50.0, 0.9)])
def test_steady_drag_velocity_on_gpu(darcy_A, fl0):
    """The closed-form fixed point of the solid closures (see the oracle pin): uniform mushy
    periodic box, u_z = phi G / (2 (1 - phi)), in FP64 and FP32 storage."""
    for precision, tol in ((inp.FP64, 1e-12), (inp.FP32, 1e-4)):
        p = inp.Params(flow_model=inp.FLOW_MRT, precision=precision, bc=[inp.PERIODIC] * 6,
                       Ra=1e5, Pr=0.7, St=1.0, darcy_A=darcy_A)
        g = LBPC((8, 5, 4), p)
        g.set_initial_h(np.full(160, fl0 * g.lattice()["latent"]))
        g.step(300)
        G = g.lattice()["gbeta"] * (0.0 - p.Tref)
        if darcy_A > 0:
            uz = G / (darcy_A * (1 - fl0) ** 2 / (fl0 ** 3 + 1e-3))
        else:
            uz = fl0 * G / (2 * (1 - fl0))
        u = _np(g.fields())["u"]
        assert np.abs(u[2] - uz).max() <= tol * abs(uz), precision


@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
def test_short_steps_before_the_first_diagnostics(streaming):
    """With report_every > 0, calls that end before the first diagnostics point report no
    divergence (nothing recorded yet) and equal stepping in one call."""
    shape = (24, 12, 10)
    p = inp.Params(precision=inp.FP32, streaming=streaming, Ra=1e5, Pr=0.7, St=1.0,
                   report_every=10)
    h0 = np.random.default_rng(2).uniform(-0.3, 1.8, int(np.prod(shape)))
    a, b = LBPC(shape, p), LBPC(shape, p)
    a.set_initial_h(h0)
    b.set_initial_h(h0)
    a.step(23)
    for _ in range(23):
        b.step(1)
    assert a.step_count == b.step_count == 23
    Fa, Fb = _np(a.fields()), _np(b.fields())
    for k in KEYS:
        assert np.array_equal(Fa[k], Fb[k]), k
    assert np.array_equal(a.history(), b.history())


@pytest.mark.parametrize("bc", [
    [inp.PERIODIC] * 6,
    [inp.ADIABATIC] * 6,
    [inp.ISOTHERMAL, inp.ADIABATIC, inp.PERIODIC, inp.PERIODIC, inp.ISOTHERMAL, inp.ADIABATIC],
])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (33, 1, 2), (5, 34, 3)])
def test_edge_shapes_and_boundaries_fp64(bc, shape):
    p = inp.Params(flow_model=inp.FLOW_MRT, precision=inp.FP64, bc=bc, Ra=1e4, Pr=1.0,
                   St=0.5, T_wall=[1.0, 0.0, 0.0, 0.0, 0.7, 0.0])
    rng = np.random.default_rng(2)
    h0 = rng.uniform(-0.5, 3.0, int(np.prod(shape)))
    g, o = _pair(shape, p, h0=h0)
    g.step(17)
    o.step(17)
    err = _maxerr(_np(g.fields()), o.fields())
    assert max(err.values()) <= 1e-11, err


def test_wall_temperature_field_fp64():
    shape = (10, 8, 6)
    p = inp.Params(flow_model=inp.FLOW_MRT, precision=inp.FP64, Ra=2e4, Pr=0.7, St=1.0)
    Tw = inp.wall_temperature_field(shape[1], shape[2], seed=3)
    g, o = _pair(shape, p, h0=np.zeros(int(np.prod(shape))), walls={0: Tw})
    g.step(80)
    o.step(80)
    err = _maxerr(_np(g.fields()), o.fields())
    assert max(err.values()) <= 1e-11, err
    sg, so = g.scalars(), o.diagnostics()
    for k in ("liquid_vol", "nu_hot", "nu_fd", "sum_h", "sum_rho", "front_mid"):
        assert abs(sg[k] - so[k]) <= 1e-10 * max(1.0, abs(so[k])), k


# ------------------------------------------------------------------------------------
# One step from a random non-equilibrium state, every storage precision
# ------------------------------------------------------------------------------------
TOL = {inp.FP64: 1e-13, inp.FP32: 5e-6, inp.FP16: 2.5e-4, inp.BF16: 2e-3, inp.FP16_G32: 2.5e-4,
       inp.BF16_G32: 2e-3}


@pytest.mark.parametrize("precision", [inp.FP64, inp.FP32, inp.FP16, inp.BF16, inp.FP16_G32,
                                       inp.BF16_G32])
@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
@pytest.mark.parametrize("flow_model", [inp.FLOW_MRT, inp.FLOW_SRT, inp.FLOW_NONE])
@pytest.mark.parametrize("nx", [19, 20])  # odd: one node per thread; even: node pairs
def test_one_step_from_random_state(precision, streaming, flow_model, nx):
    shape = (nx, 6, 5)
    p = inp.Params(flow_model=flow_model, precision=precision, streaming=streaming,
                   Ra=5e4, Pr=0.5, St=0.7, tau_g=0.0 if flow_model else 0.9,
                   bc=[inp.ISOTHERMAL, inp.ISOTHERMAL, inp.PERIODIC, inp.PERIODIC,
                       inp.ADIABATIC, inp.ADIABATIC])
    f, gq = inp.random_state(shape, seed=4, flow=flow_model != 0)
    dev = torch.device("cuda")
    g = LBPC(shape, p)
    g.set_distributions(torch.from_numpy(f).to(dev) if f is not None else None,
                        torch.from_numpy(gq).to(dev))
    f0, g0 = g.distributions()  # the state as rounded to the storage precision
    o = oracle.Oracle(shape, p)
    o.set_distributions(f0.cpu().numpy() if f0 is not None else None, g0.cpu().numpy())
    for _ in range(2):
        g.step(1)
        o.step(1)
        f1, g1 = g.distributions()
        fo, go = o.distributions()
        g1n = g1.cpu().numpy()
        assert np.abs(g1n[1:] - go[1:]).max() <= TOL[precision]
        assert np.abs(g1n[0] - go[0]).max() <= 6 * TOL[precision]
        if flow_model:
            assert np.abs(f1.cpu().numpy() - fo).max() <= TOL[precision]
        # the state the oracle continues from is the GPU's (rounded) one
        o.set_distributions(f1.cpu().numpy() if f1 is not None else None, g1.cpu().numpy())


# Rows of 256 nodes: one 128-thread block of node pairs per row, the two x faces in
# different warps of the block; x walls (isothermal: anti-bounce-back of g, bounce-back of
# f, a per-node wall field) and x periodic (the wrap crosses warps), every storage mode,
# both solid closures.
@pytest.mark.parametrize("precision", [inp.FP32, inp.FP16, inp.BF16, inp.FP16_G32, inp.BF16_G32])
@pytest.mark.parametrize("flow_model,darcy_A", [(inp.FLOW_MRT, 0.0), (inp.FLOW_SRT, 0.0),
                                                (inp.FLOW_NONE, 0.0), (inp.FLOW_MRT, 3.0)])
@pytest.mark.parametrize("xbc", [inp.ISOTHERMAL, inp.PERIODIC])
def test_one_step_from_random_state_wide_rows(precision, flow_model, darcy_A, xbc):
    shape = (256, 6, 5)
    bc = [xbc, xbc, inp.PERIODIC, inp.PERIODIC, inp.ADIABATIC, inp.ADIABATIC]
    p = inp.Params(flow_model=flow_model, precision=precision, streaming=inp.PULL, Ra=5e4,
                   Pr=0.5, St=0.7, tau_g=0.0 if flow_model else 0.9, bc=bc, darcy_A=darcy_A)
    f, gq = inp.random_state(shape, seed=6, flow=flow_model != 0)
    dev = torch.device("cuda")
    g = LBPC(shape, p)
    if xbc == inp.ISOTHERMAL:
        g.set_wall_temperature(0, inp.wall_temperature_field(6, 5, seed=2))
    g.set_distributions(torch.from_numpy(f).to(dev) if f is not None else None,
                        torch.from_numpy(gq).to(dev))
    f0, g0 = g.distributions()
    o = oracle.Oracle(shape, p)
    if xbc == inp.ISOTHERMAL:
        o.set_wall_temperature(0, inp.wall_temperature_field(6, 5, seed=2))
    o.set_distributions(f0.cpu().numpy() if f0 is not None else None, g0.cpu().numpy())
    for _ in range(3):
        g.step(1)
        o.step(1)
        f1, g1 = g.distributions()
        fo, go = o.distributions()
        g1n = g1.cpu().numpy()
        assert np.abs(g1n[1:] - go[1:]).max() <= TOL[precision]
        assert np.abs(g1n[0] - go[0]).max() <= 6 * TOL[precision]
        if flow_model:
            assert np.abs(f1.cpu().numpy() - fo).max() <= TOL[precision]
        o.set_distributions(f1.cpu().numpy() if f1 is not None else None, g1.cpu().numpy())


@pytest.mark.parametrize("precision,tol", [(inp.FP32, 1e-5), (inp.FP16, 1e-3)])
@pytest.mark.parametrize("shape", [(256, 8, 6), (512, 4, 3)])
def test_wide_row_cavity_tracks_oracle(precision, tol, shape):
    """Rows of one and of two 128-pair blocks, 300 steps of the melting cavity against the
    oracle, and the diagnostics' sum of h against the fields."""
    p = inp.Params(precision=precision, Ra=1e5, Pr=0.71, St=1.0)
    h0 = np.random.default_rng(7).uniform(-1e-6, 1e-6, int(np.prod(shape)))
    g, o = _pair(shape, p, h0=h0)
    g.step(300)
    o.step(300)
    F = _np(g.fields())
    err = _maxerr(F, o.fields(), ("T", "fl", "rho", "h"))
    assert max(err.values()) <= tol, err
    # the diagnostics reduce the GPU's own h field in FP64; against the oracle the sum can
    # differ by at most the per-node tolerance times the node count (isothermal walls let
    # FP32-rounded fluxes in and out every step)
    sg, so = g.scalars(), o.diagnostics()
    assert abs(sg["sum_h"] - F["h"].sum()) <= 1e-12 * abs(F["h"]).sum()
    assert abs(sg["sum_h"] - so["sum_h"]) <= tol * F["h"].size


@pytest.mark.parametrize("precision,tol", [(inp.FP64, 1e-13), (inp.FP32, 2e-6), (inp.FP16, 1e-3)])
def test_aa_and_pull_agree(precision, tol):
    """The two streaming schemes compute the same arithmetic on the same values; they
    differ only where the compiler contracts a multiply-add differently in the two
    kernel instantiations (FP32 rounding), which in FP16 storage can move a stored value
    by one FP16 ulp (2.4e-4 at 0.25)."""
    shape = (16, 12, 10)
    res = {}
    for streaming in (inp.PULL, inp.AA):
        p = inp.Params(precision=precision, streaming=streaming, Ra=5e4, Pr=0.7, St=1.0)
        g = LBPC(shape, p)
        g.set_initial_h(np.linspace(-0.2, 1.5, int(np.prod(shape))))
        g.step(41)
        res[streaming] = _np(g.fields())
    for k in KEYS:
        assert np.abs(res[inp.PULL][k] - res[inp.AA][k]).max() <= tol, k


@pytest.mark.parametrize("precision,tol", [(inp.FP32, 1e-5), (inp.FP16, 1e-3), (inp.BF16, 1e-2),
                                           (inp.FP16_G32, 1e-4), (inp.BF16_G32, 1e-3)])
def test_cavity_reduced_precision_tracks_oracle(precision, tol):
    shape = (24, 16, 12)
    p = inp.Params(precision=precision, Ra=1e5, Pr=0.71, St=1.0)
    rng = np.random.default_rng(5)
    h0 = rng.uniform(-1e-6, 1e-6, int(np.prod(shape)))
    g, o = _pair(shape, p, h0=h0)
    g.step(400)
    o.step(400)
    err = _maxerr(_np(g.fields()), o.fields(), ("T", "fl"))
    assert max(err.values()) <= tol, err


# ------------------------------------------------------------------------------------
# Conservation, checkpoints, diagnostics history, divergence detection
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision,rho_tol", [(inp.FP64, 1e-13), (inp.FP32, 1e-5),
                                               (inp.FP16, 2e-3), (inp.BF16, 2e-2),
                                               (inp.FP16_G32, 2e-3), (inp.BF16_G32, 2e-2)])
def test_closed_box_conserves_enthalpy_exactly(precision, rho_tol):
    """Adiabatic no-slip box with buoyancy and phase change: the FP64 rest channel makes
    sum h exact to FP64 rounding in every storage precision (Eq. 9 telescoping)."""
    shape = (17, 9, 8)
    p = inp.Params(precision=precision, bc=[inp.ADIABATIC] * 6, Ra=5e4, Pr=0.7, St=0.5)
    rng = np.random.default_rng(6)
    g = LBPC(shape, p)
    g.set_initial_h(rng.uniform(-0.5, 2.5, int(np.prod(shape))))
    s0 = g.scalars()
    g.step(500)
    s1 = g.scalars()
    assert abs(s1["sum_h"] - s0["sum_h"]) <= 1e-12 * abs(s0["sum_h"])
    assert abs(s1["sum_rho"] - s0["sum_rho"]) <= rho_tol * s0["sum_rho"]
    assert 0 < s1["liquid_vol"] < np.prod(shape)


@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
def test_save_load_continues_identically(streaming):
    shape = (12, 10, 8)
    p = inp.Params(precision=inp.FP32, streaming=streaming, Ra=5e4, Pr=0.7, St=1.0)
    g = LBPC(shape, p)
    g.set_initial_h(np.zeros(int(np.prod(shape))))
    g.step(11)
    blob = g.save()
    g.step(9)
    A = _np(g.fields())
    g2 = LBPC(shape, p)
    g2.load(blob)
    assert g2.step_count == 11
    g2.step(9)
    B2 = _np(g2.fields())
    for k in KEYS:
        assert np.array_equal(A[k], B2[k]), k


def test_history_rows_and_host_fields():
    shape = (16, 8, 8)
    p = inp.Params(precision=inp.FP32, Ra=5e4, Pr=0.7, St=1.0, report_every=5)
    g = LBPC(shape, p)
    g.step(20)
    H = g.history()
    assert H.shape == (4, len(B.S_NAMES))
    assert np.array_equal(H[:, B.S_NAMES.index("step")], [5, 10, 15, 20])
    s = g.scalars()
    assert np.allclose(H[-1], [s[k] for k in B.S_NAMES], rtol=0, atol=0)
    Fd, Fh = _np(g.fields()), g.fields_host()
    for k in KEYS:
        assert np.array_equal(Fd[k], Fh[k]), k


@pytest.mark.parametrize("flow_model", [inp.FLOW_MRT, inp.FLOW_NONE])
def test_divergence_is_reported_and_blocks_stepping(flow_model):
    shape = (8, 8, 8)
    p = inp.Params(flow_model=flow_model, precision=inp.FP32, Ra=5e4, Pr=0.7, St=1.0,
                   tau_g=0.0 if flow_model else 0.9, report_every=1)
    g = LBPC(shape, p)
    f, gq = inp.random_state(shape, seed=7, flow=flow_model != 0)
    if flow_model:
        f[3, 100] = np.nan  # a host-made bad state; no device fault involved
    else:
        gq[5, 100] = np.nan
    dev = torch.device("cuda")
    g.set_distributions(torch.from_numpy(f).to(dev) if f is not None else None,
                        torch.from_numpy(gq).to(dev))
    with pytest.raises(LbpcError) as e:
        g.step(2)
    assert e.value.status == B.LBPC_ERR_DIVERGED
    assert g.scalars()["nan"] >= 1
    with pytest.raises(LbpcError) as e2:
        g.step(1)
    assert e2.value.status == B.LBPC_ERR_STATE
    g.set_initial_h(np.zeros(512))
    g.step(1)


@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
@pytest.mark.parametrize("precision", [inp.FP32, inp.FP16])
@pytest.mark.parametrize("flow_model", [inp.FLOW_MRT, inp.FLOW_NONE])
def test_divergence_is_reported_without_diagnostics(streaming, precision, flow_model):
    """report_every = 0: no diagnostics are recorded, and each stepping call checks the
    FP64 rest channel once at its end.  A host-made non-finite population (of f, or of g
    in a conduction-only run) reaches it within one step."""
    shape = (10, 6, 5)
    p = inp.Params(flow_model=flow_model, precision=precision, streaming=streaming, Ra=5e4,
                   Pr=0.7, St=1.0, tau_g=0.0 if flow_model else 0.9, report_every=0)
    g = LBPC(shape, p)
    g.step(4)  # a finite state passes the check (AA: even, so a state can be loaded)
    f, gq = inp.random_state(shape, seed=8, flow=flow_model != 0)
    if flow_model:
        f[7, 41] = np.inf
    else:
        gq[3, 41] = np.nan
    dev = torch.device("cuda")
    g.set_distributions(torch.from_numpy(f).to(dev) if f is not None else None,
                        torch.from_numpy(gq).to(dev))
    launches = g.launch_count
    with pytest.raises(LbpcError) as e:
        g.step(2)
    assert e.value.status == B.LBPC_ERR_DIVERGED
    assert g.launch_count == launches + 3  # two steps and one check
    with pytest.raises(LbpcError) as e2:
        g.step(1)
    assert e2.value.status == B.LBPC_ERR_STATE
    g.set_initial_h(np.zeros(int(np.prod(shape))))
    g.step(1)


def test_workspace_too_small_on_device():
    import ctypes as C
    p = inp.Params(precision=inp.FP32)
    cp = B.to_c(p)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    st = B.lib().lbpc_create(8, 8, 8, C.byref(cp), C.c_void_p(small.data_ptr()), 1024, None,
                             C.byref(h))
    assert st == B.LBPC_ERR_WORKSPACE
    host = np.zeros(1 << 20, dtype=np.uint8)
    st = B.lib().lbpc_create(8, 8, 8, C.byref(cp), C.c_void_p(host.ctypes.data), host.size,
                             None, C.byref(h))
    assert st == B.LBPC_ERR_WORKSPACE


# ------------------------------------------------------------------------------------
# Full size: the timed 256^3 configuration, sampled against the oracle node by node
# ------------------------------------------------------------------------------------
def _sample_nodes(shape, count, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    idx = list(rng.choice(nx * ny * nz, size=count, replace=False))
    for x in (0, nx - 1):  # corners and edges, where every wall rule meets
        for y in (0, ny - 1):
            for z in (0, nz - 1):
                idx.append(x + nx * (y + ny * z))
    for k in range(64):
        idx.append(0 + nx * (k % ny + ny * ((7 * k) % nz)))
        idx.append(nx - 1 + nx * ((3 * k) % ny + ny * (k % nz)))
    return np.unique(np.array(idx, dtype=np.int64))


@pytest.mark.parametrize("precision,tol", [(inp.FP32, 5e-6), (inp.FP16, 1e-4)])
def test_full_size_bench_configuration_sampled(precision, tol):
    w = inp.bench_workload()
    p = w.params.replace(precision=precision, report_every=0)
    g = LBPC(w.shape, p)
    g.set_initial_h(inp.h0_field(w))
    g.step(24)
    f0, g0 = g.distributions()
    f0h, g0h = f0.cpu().numpy(), g0.cpu().numpy()
    del f0, g0
    g.step(1)
    f1, g1 = g.distributions()
    idx = _sample_nodes(w.shape, 4000, seed=8)
    it = torch.from_numpy(idx).cuda()
    f1s = f1[:, it].cpu().numpy().T
    g1s = g1[:, it].cpu().numpy().T
    del f1, g1
    o = oracle.Oracle(w.shape, p, alloc=False)
    fo, go = o.update_sampled(f0h, g0h, idx)
    assert np.abs(f1s - fo).max() <= tol
    assert np.abs(g1s - go).max() <= tol
    s = g.scalars()
    assert s["nan"] == 0 and s["liquid_vol"] > 0


def test_lattice_above_the_pair_limit():
    """A lattice of 1024 x 1024 x 684 = 717,225,984 nodes (above (2^31 - 1)/3, so the step runs
    the one-node-per-thread kernels; FP16 storage with flow, 83 GB of workspace), periodic,
    with an enthalpy that varies only along z: every (x, y) column must then evolve exactly
    like the 1 x 1 x 684 oracle lattice, which any index error at this size would break."""
    shape = (1024, 1024, 684)
    nx, ny, nz = shape
    p = inp.Params(flow_model=inp.FLOW_MRT, precision=inp.FP16, bc=[inp.PERIODIC] * 6, Ra=1e5,
                   Pr=0.7, St=1.0, report_every=0)
    o = oracle.Oracle((1, 1, nz), p)
    L = o.lattice()["latent"]
    z = np.arange(nz)
    hz = L + 0.5 + 0.3 * np.sin(2 * np.pi * z / nz)  # liquid, T between 0.2 and 0.8
    o.set_initial_h(hz)
    o.step(3)
    Tz = o.fields()["T"][:, 0, 0]
    g = LBPC(shape, p)
    g.set_initial_h(np.repeat(hz, nx * ny))
    g.step(3)
    F = g.fields()
    T = F["T"]
    del F
    rng = np.random.default_rng(4)
    xs = np.concatenate([[0, nx - 1], rng.integers(0, nx, 64)])
    ys = np.concatenate([[0, ny - 1], rng.integers(0, ny, 64)])
    for zz in (0, nz // 2, nz - 1):
        plane = T[zz, :, :]
        assert float((plane.max() - plane.min()).item()) < 1e-12  # uniform in x and y
        assert abs(float(plane[ys[0], xs[0]].item()) - Tz[zz]) < 2e-3
    Tc = T[:, ys[2], xs[2]].cpu().numpy()  # one column against the oracle
    assert np.abs(Tc - Tz).max() < 2e-3
    del T
    assert g.scalars()["nan"] == 0
