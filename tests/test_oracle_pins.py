"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not compute itself: the
polynomial definitions of the moment bases (d'Humieres et al. 2002, the paper's
Ref. [20] for Eq. 51; Eq. 24), the textbook D3Q19 equilibrium and discrete forcing
(whose moments Eq. 53 / 54 must be), the moment relations the paper states
(Eq. 9, Eq. 7 vs Eq. 25), exact conservation, invariance of the rest state and
mirror symmetry.
"""
import numpy as np
import pytest

import lbpc_inputs as inp
import oracle

M, MINV, NM, NINV, E19, E7 = oracle.tables()
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _opp(e):
    return np.array([int(np.where((e == -e[a]).all(axis=1))[0][0]) for a in range(len(e))])


def test_velocity_sets():
    # Eq. 3 and Eq. 4 for D3Q7
    assert E7.shape == (7, 3)
    assert np.all(E7.sum(axis=0) == 0)
    assert np.array_equal(E7.T @ E7, 2 * np.eye(3, dtype=int))
    # Eq. 48: 19 distinct vectors, rest + 6 axis + 12 face diagonals, closed under negation
    assert len({tuple(v) for v in E19}) == 19
    norms = (E19 ** 2).sum(axis=1)
    assert sorted(norms.tolist()) == [0] + [1] * 6 + [2] * 12
    assert np.array_equal(E19[_opp(E19)], -E19)
    # standard D3Q19 isotropy with weights 1/3, 1/18, 1/36
    assert np.isclose(W19.sum(), 1)
    assert np.allclose((W19[:, None, None] * E19[:, :, None] * E19[:, None, :]).sum(0),
                       np.eye(3) / 3)


def test_flow_transform_rows_are_the_moment_polynomials():
    """Eq. 51 as transcribed equals the d'Humieres polynomial basis of e."""
    ex, ey, ez = (E19[:, d].astype(float) for d in range(3))
    e2 = ex ** 2 + ey ** 2 + ez ** 2
    rows = [np.ones(19), 19 * e2 - 30, (21 * e2 ** 2 - 53 * e2 + 24) / 2,
            ex, (5 * e2 - 9) * ex, ey, (5 * e2 - 9) * ey, ez, (5 * e2 - 9) * ez,
            3 * ex ** 2 - e2, (3 * e2 - 5) * (3 * ex ** 2 - e2),
            ey ** 2 - ez ** 2, (3 * e2 - 5) * (ey ** 2 - ez ** 2),
            ex * ey, ey * ez, ex * ez,
            (ey ** 2 - ez ** 2) * ex, (ez ** 2 - ex ** 2) * ey, (ex ** 2 - ey ** 2) * ez]
    assert np.array_equal(M, np.array(rows))


def test_enthalpy_transform_rows():
    """Eq. 24: rows are 1, e_x, e_y, e_z, 6 - 7|e|^2, 3 e_x^2 - |e|^2, e_y^2 - e_z^2."""
    ex, ey, ez = (E7[:, d].astype(float) for d in range(3))
    e2 = ex ** 2 + ey ** 2 + ez ** 2
    rows = [np.ones(7), ex, ey, ez, 6 - 7 * e2, 3 * ex ** 2 - e2, ey ** 2 - ez ** 2]
    assert np.array_equal(NM, np.array(rows))


def test_transforms_invert_and_are_orthogonal():
    assert np.allclose(M @ MINV, np.eye(19), atol=1e-15, rtol=0)
    assert np.allclose(NM @ NINV, np.eye(7), atol=1e-15, rtol=0)
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.array_equal(np.diag(G), [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24,
                                       4, 4, 4, 8, 8, 8])
    GN = NM @ NM.T
    assert np.allclose(GN, np.diag([7, 2, 2, 2, 42, 12, 4]))


def _feq_textbook(rho, u):
    eu = E19 @ u
    return W19 * rho * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u @ u)


def _guo_textbook(F, u):
    eu = E19 @ u
    return W19 * (3 * (E19 - u) @ F + 9 * eu * (E19 @ F))


@pytest.mark.parametrize("seed", range(5))
def test_meq_is_the_moment_of_the_second_order_equilibrium(seed):
    """Eq. 53 (with element 10 as -u_x^2 + u_y^2/2 + u_z^2/2) equals M f^eq."""
    rng = np.random.default_rng(seed)
    rho, u = 1 + 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(3)
    assert np.allclose(M @ _feq_textbook(rho, u), oracle.flow_meq(rho, u), atol=1e-14, rtol=0)


@pytest.mark.parametrize("seed", range(5))
def test_forcing_moments_are_the_moments_of_the_discrete_force(seed):
    """Eq. 54 (with element 9 as 6 F_x u_x - 2 F.u) equals M applied to the
    second-order discrete forcing w_a [3 (e - u).F + 9 (e.u)(e.F)]."""
    rng = np.random.default_rng(100 + seed)
    F, u = 1e-3 * rng.standard_normal(3), 0.1 * rng.standard_normal(3)
    assert np.allclose(M @ _guo_textbook(F, u), oracle.flow_forcing(F, u), atol=1e-16, rtol=0)


def _node_oracle(**kw):
    p = inp.Params(**kw)
    return oracle.Oracle((1, 1, 1), p, alloc=False)


def test_enthalpy_equilibrium_moments():
    """Eq. 9: zeroth, first and second moments of g^eq, and N g^eq = n^eq (Eq. 25)."""
    o = _node_oracle(flow_model=0, tau_g=0.8, Cp_s=1.3, Cp_l=2.1, Cp_ref=1.7, omega_T=0.3)
    rng = np.random.default_rng(7)
    for _ in range(5):
        h, T, fl = rng.uniform(-2, 3), rng.uniform(-1, 1), rng.uniform(0, 1)
        u = 0.05 * rng.standard_normal(3)
        geq = o.enth_geq(h, T, fl, u)
        cp = fl * 2.1 + (1 - fl) * 1.3
        assert np.isclose(geq.sum(), h, atol=1e-14, rtol=0)
        assert np.allclose(E7.T @ geq, cp * T * u, atol=1e-15, rtol=0)
        second = (geq[:, None, None] * E7[:, :, None] * E7[:, None, :]).sum(0)
        assert np.allclose(second, 1.7 * T * 0.3 * np.eye(3), atol=1e-15, rtol=0)
        assert np.allclose(NM @ geq, o.enth_neq(h, T, fl, u), atol=1e-14, rtol=0)


def test_inversion_branches_of_eq2():
    """Eq. 2: h = C_p T + f_l L on each branch, continuous at both kinks."""
    o = _node_oracle(flow_model=0, tau_g=0.8, St=0.5, Cp_s=1.0, Cp_l=1.0, Tm=0.0)
    lat = o.lattice()
    L = lat["latent"]
    assert np.isclose(L, 2.0)
    for h in np.linspace(-1.5, 4.5, 61):
        T, fl = o.invert(h)
        assert 0.0 <= fl <= 1.0
        assert np.isclose(T * 1.0 + fl * L, h, atol=1e-14)
    assert o.invert(0.0) == (0.0, 0.0)
    assert o.invert(L) == (0.0, 1.0)


def _liquid_node(seed, flow_model):
    o = _node_oracle(flow_model=flow_model, Ra=1e4, Pr=0.7, St=1.0)
    rng = np.random.default_rng(seed)
    f = W19 * (1 + 0.2 * rng.uniform(-1, 1, 19))
    g = np.empty(7)
    g[1:] = rng.uniform(0.05, 0.2, 6)
    g[0] = o.lattice()["hl"] + 0.7 - g[1:].sum()  # liquid: h = h_l + 0.7
    return o, f, g


@pytest.mark.parametrize("seed", range(3))
def test_mrt_flow_with_one_rate_is_bgk_with_discrete_forcing(seed):
    """With every relaxation rate equal to 1/tau (the SRT variant), Eq. 49-50 must
    reduce to BGK with the second-order discrete forcing, written here in velocity space.
    Eq. 56 divides by rho_0 while Eq. 53 multiplies by rho; the two agree (and BGK
    conserves momentum) only on a node with rho = rho_0 = 1, so the node is normalised."""
    o, f, g = _liquid_node(seed, inp.FLOW_SRT)
    f = f / f.sum()
    fp, _, mac = o.collide_node(f, g)
    lat = o.lattice()
    tau = lat["tau_f"]
    rho = f.sum()
    j = E19.T @ f
    F = np.array([0.0, 0.0, lat["gbeta"] * (mac["T"] - 0.5)])
    u = j + 0.5 * F
    assert mac["fl"] == 1.0
    ref = f - (f - _feq_textbook(rho, u)) / tau + (1 - 0.5 / tau) * _guo_textbook(F, u)
    assert np.allclose(fp, ref, atol=1e-15, rtol=0)


@pytest.mark.parametrize("tau", [0.564, 0.8, 1.0, 1.6])
def test_mrt_enthalpy_with_one_rate_equals_srt(tau):
    """Eq. 21 with R = I/tau_g must equal the BGK update Eq. 5-6."""
    rng = np.random.default_rng(3)
    g = np.concatenate([[0.4], rng.uniform(0, 0.2, 6)])
    u = np.zeros(3)
    o_srt = _node_oracle(flow_model=0, enth_model=inp.ENTH_SRT, tau_g=tau, St=0.3)
    o_mrt = _node_oracle(flow_model=0, enth_model=inp.ENTH_MRT, tau_g=tau, St=0.3,
                         sigma4=1 / tau)
    _, gs, _ = o_srt.collide_node(None, g)
    _, gm, _ = o_mrt.collide_node(None, g)
    assert np.allclose(gs, gm, atol=1e-14, rtol=0)
    if tau == 1.0:  # tau = 1: post-collision state is the equilibrium
        mac = o_srt.collide_node(None, g)[2]
        assert np.allclose(gs, o_srt.enth_geq(mac["h"], mac["T"], mac["fl"], u), atol=1e-15)


def test_solid_node_keeps_zero_velocity():
    """Solid-phase forcing: in a fully solid node the velocity of Eq. 56 is zero and
    the collision reverses the momentum exactly."""
    o = _node_oracle(flow_model=inp.FLOW_MRT, Ra=1e5, Pr=0.02, St=1.0)
    rng = np.random.default_rng(11)
    f = W19 * (1 + 0.1 * rng.uniform(-1, 1, 19))
    g = np.concatenate([[-0.3], np.zeros(6)])  # h = -0.3 < h_s = 0: solid
    fp, _, mac = o.collide_node(f, g)
    assert mac["fl"] == 0.0
    assert np.allclose(mac["u"], 0.0, atol=1e-17)
    assert np.allclose(E19.T @ fp, -(E19.T @ f), atol=1e-15)
    assert np.isclose(fp.sum(), f.sum(), atol=1e-15)


def _cavity_params(**kw):
    base = dict(flow_model=inp.FLOW_MRT, enth_model=inp.ENTH_MRT, Ra=1e4, Pr=1.0, St=1.0,
                precision=inp.FP64)
    base.update(kw)
    return inp.Params(**base)


def test_rest_state_is_invariant():
    """Uniform rho = 1, u = 0, all liquid at T = T_ref (no buoyancy), walls at T_ref:
    the state must not change."""
    p = _cavity_params(T_wall=[0.5, 0.5, 0, 0, 0, 0])
    o = oracle.Oracle((6, 5, 4), p)
    L = o.lattice()["latent"]
    o.set_initial_h(np.full(o.N, L + 0.5))
    f0, g0 = o.distributions()
    o.step(40)
    f1, g1 = o.distributions()
    # FP64 rounding only: a few ulp of the largest population (g_0 ~ 1.1) over 40 steps
    assert np.abs(f1 - f0).max() <= 1e-14
    assert np.abs(g1 - g0).max() <= 1e-14


@pytest.mark.parametrize("flow_model,enth_model", [(inp.FLOW_MRT, inp.ENTH_MRT),
                                                   (inp.FLOW_SRT, inp.ENTH_SRT)])
def test_closed_adiabatic_box_conserves_enthalpy_and_mass(flow_model, enth_model):
    """All faces adiabatic and no-slip: streaming with bounce-back is a permutation and
    both collisions conserve their zeroth moment, so sum h and sum rho stay fixed
    (buoyancy and phase change both active)."""
    p = _cavity_params(flow_model=flow_model, enth_model=enth_model,
                       bc=[inp.ADIABATIC] * 6)
    o = oracle.Oracle((9, 7, 6), p)
    rng = np.random.default_rng(5)
    o.set_initial_h(rng.uniform(-0.5, 2.5, o.N))  # solid, mushy and liquid nodes
    d0 = o.diagnostics()
    o.step(300)
    d1 = o.diagnostics()
    assert abs(d1["sum_h"] - d0["sum_h"]) <= 1e-12 * abs(d0["sum_h"])
    assert abs(d1["sum_rho"] - d0["sum_rho"]) <= 1e-12 * d0["sum_rho"]
    assert 0 < d1["liquid_vol"] < o.N
    assert np.abs(o.fields()["u"]).max() > 1e-6  # the flow was driven


def test_mirror_symmetry_in_y():
    """Cavity with hot and cold x walls and gravity along -z: the solution is symmetric
    under y -> ny - 1 - y with u_y changing sign."""
    p = _cavity_params()
    o = oracle.Oracle((10, 7, 6), p)
    o.set_initial_h(np.zeros(o.N))
    o.step(300)
    F = o.fields()
    assert F["fl"].sum() > 1
    for k in ("T", "fl", "h", "rho"):
        assert np.abs(F[k] - F[k][:, ::-1, :]).max() <= 1e-12, k
    u = F["u"]
    assert np.abs(u[0] - u[0][:, ::-1, :]).max() <= 1e-12
    assert np.abs(u[1] + u[1][:, ::-1, :]).max() <= 1e-12
    assert np.abs(u[2] - u[2][:, ::-1, :]).max() <= 1e-12
    assert np.abs(u).max() > 1e-5


@pytest.mark.parametrize("darcy_A,fl0", [(0.0, 0.3), (0.0, 0.9), (1.0, 0.3), (50.0, 0.9)])
def test_solid_closures_reach_the_steady_drag_velocity(darcy_A, fl0):
    """Uniform mushy periodic box at T_m: buoyancy is a uniform body force G = g beta (T_m -
    T_ref) along z, and each step adds F = G + F_s to the momentum.  With u = phi u* and F_s =
    -2 (1 - phi) u* the fixed point is u* = G / (2 (1 - phi)), u_z = phi G / (2 (1 - phi)):
    phi = f_l for the liquid-fraction closure (Sec. 3.3 reading), and for the enthalpy-porosity
    drag phi = 1 / (1 + D/2), D = A (1 - f_l)^2 / (f_l^3 + 1e-3), i.e. u_z = G / D."""
    p = inp.Params(flow_model=inp.FLOW_MRT, precision=inp.FP64, bc=[inp.PERIODIC] * 6,
                   Ra=1e5, Pr=0.7, St=1.0, darcy_A=darcy_A)
    o = oracle.Oracle((6, 5, 4), p)
    o.set_initial_h(np.full(o.N, fl0 * o.lattice()["latent"]))
    o.step(300)
    F = o.fields()
    G = o.lattice()["gbeta"] * (0.0 - p.Tref)
    if darcy_A > 0:
        D = darcy_A * (1 - fl0) ** 2 / (fl0 ** 3 + 1e-3)
        uz = G / D
    else:
        uz = fl0 * G / (2 * (1 - fl0))
    assert np.abs(F["u"][2] - uz).max() <= 1e-12 * abs(uz)
    assert np.abs(F["u"][:2]).max() <= 1e-15
    assert np.abs(F["fl"] - fl0).max() == 0.0


_SAMPLED_CASES = [
    # (shape, bc of the six faces, flow model, enthalpy model, enthalpy-porosity A)
    ((1, 1, 1), [inp.PERIODIC] * 6, inp.FLOW_MRT, inp.ENTH_MRT, 0.0),
    ((1, 1, 1), [inp.ISOTHERMAL, inp.ADIABATIC, inp.ADIABATIC, inp.ISOTHERMAL,
                 inp.ISOTHERMAL, inp.ADIABATIC], inp.FLOW_MRT, inp.ENTH_MRT, 0.0),
    ((3, 2, 5), [inp.ISOTHERMAL, inp.ISOTHERMAL, inp.ADIABATIC, inp.ADIABATIC,
                 inp.ADIABATIC, inp.ADIABATIC], inp.FLOW_MRT, inp.ENTH_MRT, 0.0),
    ((3, 2, 5), [inp.ISOTHERMAL, inp.ADIABATIC, inp.PERIODIC, inp.PERIODIC,
                 inp.ADIABATIC, inp.ISOTHERMAL], inp.FLOW_SRT, inp.ENTH_SRT, 0.0),
    ((6, 5, 4), [inp.PERIODIC, inp.PERIODIC, inp.ISOTHERMAL, inp.ADIABATIC,
                 inp.ISOTHERMAL, inp.ISOTHERMAL], inp.FLOW_MRT, inp.ENTH_SRT, 0.0),
    ((6, 5, 4), [inp.ADIABATIC, inp.ISOTHERMAL, inp.ISOTHERMAL, inp.ISOTHERMAL,
                 inp.PERIODIC, inp.PERIODIC], inp.FLOW_SRT, inp.ENTH_MRT, 0.0),
    ((5, 4, 3), [inp.ISOTHERMAL, inp.ISOTHERMAL, inp.ADIABATIC, inp.ADIABATIC,
                 inp.ADIABATIC, inp.ADIABATIC], inp.FLOW_MRT, inp.ENTH_MRT, 5.0),
    ((4, 3, 7), [inp.ISOTHERMAL, inp.ADIABATIC, inp.ISOTHERMAL, inp.ADIABATIC,
                 inp.PERIODIC, inp.PERIODIC], inp.FLOW_NONE, inp.ENTH_MRT, 0.0),
    ((7, 1, 2), [inp.ISOTHERMAL, inp.ISOTHERMAL, inp.PERIODIC, inp.PERIODIC,
                 inp.PERIODIC, inp.PERIODIC], inp.FLOW_NONE, inp.ENTH_SRT, 0.0),
]


@pytest.mark.parametrize("case", range(len(_SAMPLED_CASES)))
def test_sampled_update_equals_the_full_step(case):
    """The node-by-node update (used to check single nodes of lattices too large for a
    full oracle step) must give the post-stream populations of one full step exactly.
    It rebuilds the pull stream of Eq. 5 / Eq. 50 and the half-way wall rules
    (bounce-back of f and of g on adiabatic faces, anti-bounce-back -g*_abar +
    omega_T C_p,ref T_w on isothermal faces) on its own, one node at a time, so a wrong
    face, upwind index or opposite slot there differs from the full step at some node.
    Every lattice here reaches each rule it has: periodic wraps, all six face kinds, edges
    and corners, per-node wall temperatures, extents of one node."""
    shape, bc, flow_model, enth_model, darcy_A = _SAMPLED_CASES[case]
    rng = np.random.default_rng(40 + case)
    T_wall = list(rng.uniform(-0.5, 1.5, 6))
    p = inp.Params(flow_model=flow_model, enth_model=enth_model, precision=inp.FP64, bc=bc,
                   T_wall=T_wall, Ra=1e5, Pr=0.7, St=1.0, darcy_A=darcy_A,
                   tau_g=0.8 if flow_model == inp.FLOW_NONE else 0.0)
    o = oracle.Oracle(shape, p)
    nx, ny, nz = shape
    area = [ny * nz, ny * nz, nx * nz, nx * nz, nx * ny, nx * ny]
    for face in range(6):
        if bc[face] == inp.ISOTHERMAL and face % 2 == case % 2:
            o.set_wall_temperature(face, rng.uniform(-0.5, 1.5, area[face]))
    f, g = inp.random_state(shape, seed=case, flow=o.flow)
    o.set_distributions(f, g)
    f0, g0 = o.distributions()
    everywhere = np.arange(o.N)
    fo, go = o.update_sampled(f0, g0, everywhere)
    some = rng.integers(0, o.N, size=2 * o.N + 3)  # random order, with repeats
    fs, gs = o.update_sampled(f0, g0, some)
    o.step(1)
    f1, g1 = o.distributions()
    assert np.array_equal(go, g1.T)
    assert np.array_equal(gs, g1.T[some])
    if o.flow:
        assert np.array_equal(fo, f1.T)
        assert np.array_equal(fs, f1.T[some])
    # the step changed the state, so equality is not a copy of the input
    assert np.abs(g1 - g0).max() > 1e-3
