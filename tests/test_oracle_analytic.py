"""Pins of the oracle against closed forms and the paper's printed numbers.

* Eq. 61: the melting root reproduces the interface position the paper prints.
* Eq. 60-61: 1D melting of a half-space (the 64x4x4 conduction workload).
* Eq. 62-63: 1D solidification, Sec. 3.1.2 cases (a) and (b) (per-phase C_p and lambda).
* Eq. 20 / Eq. 34: the decay rate of a sinusoidal conduction mode gives back the
  diffusivity fixed by the relaxation time.
* Eq. 47 (Sec. 2.4): with sigma_1 + sigma_4 = 2 the solid ahead of the front stays
  exactly at h_m; otherwise it does not; SRT with tau far from 1 cools the solid.
* The relaxation-time study of Sec. 3.1.1 (SRT vs MRT at tau = 0.564, 1.012, 6.9) and the
  rule-breaking cases (c)/(d) of Sec. 3.1.2, as the paper describes them.
* Quasi-2D convective melting (Sec. 3.2.2): the conduction limit at early Fo (Eq. 61) and
  the convective bending of the interface later.
* 2D corner solidification (Sec. 3.2.1): diagonal symmetry, the 1D Neumann limit far from
  the corner, self-similar corner enhancement.
* Steady conduction between isothermal walls gives Nu = 1.
"""
import math
import os

import numpy as np
import pytest

import lbpc_inputs as inp
import oracle
from oracle import neumann as nm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_melting_root_reproduces_printed_front():
    rows = np.loadtxt(os.path.join(GOLDEN, "neumann_melting_front.txt"), ndmin=2)
    for chi, ste, t, X in rows:
        k = nm.melting_k(ste)
        assert abs(float(nm.melting_front(t, chi, k)) - X) < 5e-4
        # the root satisfies Eq. 61 itself
        assert abs(ste / (math.exp(k * k) * math.erf(k)) - k * math.sqrt(math.pi)) < 1e-12


def test_solidification_root_case_a():
    # equal properties: Ste_s = Ste_l = 0.004, chi_s = chi_l
    k = nm.solidification_k(0.004, 0.004, 0.4, 0.4)
    # small-k limit of Eq. 63 with equal properties: Ste/(k sqrt(pi)) ... solved exactly
    lhs = 0.004 / (math.exp(k * k) * math.erf(k)) - 0.004 / (math.exp(k * k) * math.erfc(k))
    assert abs(lhs - k * math.sqrt(math.pi)) < 1e-12
    assert 0.043 < k < 0.044


@pytest.mark.parametrize("enth_model,tol", [(inp.ENTH_MRT, 0.01), (inp.ENTH_SRT, 0.03)])
def test_stefan_melting_front_and_profile(enth_model, tol):
    """64x4x4, St = 0.1, tau_g = 0.8 (chi = 0.075), 5000 steps, hot wall at x = -1/2."""
    w = inp.stefan_melting(enth_model=enth_model)
    o = oracle.run(w)
    lat = o.lattice()
    assert np.isclose(lat["chi"], 0.075)
    k = nm.melting_k(0.1)
    X = float(nm.melting_front(w.steps, lat["chi"], k))
    d = o.diagnostics()
    assert abs(d["front_mean"] - X) / X < tol
    F = o.fields()
    T = F["T"][0, 0, :]
    x = np.arange(w.shape[0]) + 0.5
    Ta = nm.melting_temperature(x, w.steps, lat["chi"], k)
    liquid = F["fl"][0, 0, :] == 1.0
    assert np.abs(T[liquid] - Ta[liquid]).max() < (0.01 if enth_model == inp.ENTH_MRT else 0.03)
    # uniform in y and z
    assert np.abs(F["T"] - F["T"][:1, :1, :]).max() < 1e-14


def test_stefan_solidification_case_a():
    """Sec. 3.1.2 case (a): chi = 0.4, Ste = 0.004, liquid at T0 = 1, wall at T1 = -1."""
    w = inp.stefan_solidification(nx=160)
    o = oracle.run(w)
    lat = o.lattice()
    assert np.isclose(lat["chi"], 0.4)
    k = nm.solidification_k(0.004, 0.004, 0.4, 0.4)
    t = w.steps
    X = float(nm.solidification_front(t, 0.4, k))
    F = o.fields()
    solid_depth = (1.0 - F["fl"][0, 0, :]).sum()
    assert abs(solid_depth - X) / X < 0.03
    x = np.arange(w.shape[0]) + 0.5
    Ta = nm.solidification_temperature(x, t, 0.4, 0.4, k)
    assert np.abs(F["T"][0, 0, :] - Ta).max() < 0.01


def test_solidification_root_case_b():
    # Sec. 3.1.2 case (b): Ste_s = 0.004, Ste_l = 0.008, chi_s / chi_l = (0.6/1) / (0.15/2) = 8
    k = nm.solidification_k(0.004, 0.008, 0.6, 0.075)
    r = math.sqrt(8.0)
    lhs = 0.004 / (math.exp(k * k) * math.erf(k)) - 0.008 / r / (
        math.exp(k * k * 8.0) * math.erfc(k * r))
    assert abs(lhs - k * math.sqrt(math.pi)) < 1e-12
    assert abs(k - 0.0437895) < 5e-7
    # only the ratio of the diffusivities enters k
    assert abs(nm.solidification_k(0.004, 0.008, 1.0, 0.125) - k) < 1e-12


def test_per_phase_conductivity_reduces_to_one_conductivity():
    """lambda_s = lambda_l = lambda gives the constant-rate model with tau_g =
    lambda / (omega_T C_p,ref) + 1/2 (Eq. 34 with chi = lambda / C_p,ref)."""
    w = inp.stefan_solidification_b(nx=24, ny=2, nz=2, lambda_s=0.3)
    h0 = inp.h0_field(w)
    a = w.params.replace(lambda_l=0.3)
    b = w.params.replace(lambda_s=0.0, lambda_l=0.0, tau_g=0.3 / 0.25 + 0.5)
    res = []
    for p in (a, b):
        o = oracle.Oracle(w.shape, p)
        o.set_initial_h(h0)
        o.step(400)
        res.append(o.fields())
    assert np.abs(res[0]["T"] - res[1]["T"]).max() < 1e-13
    assert np.abs(res[0]["h"] - res[1]["h"]).max() < 1e-10


def test_stefan_solidification_case_b():
    """Sec. 3.1.2 case (b): C_p,l = 2 C_p,s, lambda_s = 4 lambda_l (chi_s = 8 chi_l), Ste_s =
    0.004, Ste_l = 0.008, per-node rates from f_l.  Lattice: lambda_s = 1 (chi_s = 1,
    chi_l = 1/8), 256 nodes.  The front trails the Neumann solution (Eq. 63) by a fixed
    fraction of a cell -- the rate jumps from node to node at the front -- so its relative
    error shrinks as the front advances; the liquid temperature follows Eq. 62."""
    w = inp.stefan_solidification_b(nx=256, lambda_s=1.0)
    o = oracle.Oracle(w.shape, w.params)
    o.set_initial_h(inp.h0_field(w))
    chi_s, chi_l = 1.0, 0.125
    k = nm.solidification_k(0.004, 0.008, chi_s, chi_l)
    x = np.arange(w.shape[0]) + 0.5
    errs = []
    for t in (10000, 20000):
        o.step(t - int(o.diagnostics()["step"]))
        F = o.fields()
        X = float(nm.solidification_front(t, chi_s, k))
        depth = (1.0 - F["fl"][0, 0, :]).sum()
        errs.append((depth - X) / X)
        assert X - depth < 0.7  # lag below one cell
        Ta = nm.solidification_temperature(x, t, chi_s, chi_l, k)
        liquid = (x > X + 3) & (x < X + 4 * math.sqrt(chi_l * t))
        assert np.abs(F["T"][0, 0, liquid] - Ta[liquid]).max() < 0.01
    assert abs(errs[1]) < 0.04 and abs(errs[1]) < abs(errs[0])


def _decay_rate(nx, params, t1=300, t2=900):
    o = oracle.Oracle((nx, 1, 1), params)
    L = o.lattice()["latent"]
    x = np.arange(nx)
    amp = 0.1
    o.set_initial_h(L + 1.0 + amp * np.sin(2 * np.pi * x / nx))  # all liquid
    o.step(t1)
    a1 = abs(np.fft.rfft(o.fields()["T"][0, 0, :])[1])
    o.step(t2 - t1)
    a2 = abs(np.fft.rfft(o.fields()["T"][0, 0, :])[1])
    return math.log(a1 / a2) / (t2 - t1), o.lattice()["chi"]


@pytest.mark.parametrize("enth_model,tau", [(inp.ENTH_SRT, 0.6), (inp.ENTH_SRT, 0.8),
                                            (inp.ENTH_SRT, 1.5), (inp.ENTH_MRT, 0.6),
                                            (inp.ENTH_MRT, 0.9), (inp.ENTH_MRT, 1.4)])
def test_sine_mode_decay_gives_the_diffusivity(enth_model, tau):
    """Eq. 20 (SRT) and Eq. 34 (MRT): a periodic sine mode of T decays at chi k^2 to
    leading order; Richardson extrapolation of r/k^2 over two wavelengths removes
    the O(k^2) lattice correction."""
    p = inp.Params(flow_model=0, enth_model=enth_model, tau_g=tau, bc=[inp.PERIODIC] * 6,
                   St=1.0)
    r1, chi = _decay_rate(32, p)
    r2, _ = _decay_rate(64, p, t1=600, t2=2600)
    R1, R2 = r1 / (2 * np.pi / 32) ** 2, r2 / (2 * np.pi / 64) ** 2
    chi_ext = (4 * R2 - R1) / 3
    assert np.isclose(chi, (tau - 0.5) * 0.25)
    assert abs(R2 - chi) / chi < 0.02
    assert abs(chi_ext - chi) / chi < 1e-3


def _solid_ahead_error(w, steps):
    o = oracle.run(w, steps=steps)
    F = o.fields()
    fl = F["fl"][0, 0, :]
    h = F["h"][0, 0, :]
    front = int(np.argmax(fl < 1.0))  # first not fully liquid node
    return np.abs(h[front + 2:] - 0.0).max(), F["T"][0, 0, front + 2:].min()


def test_relaxation_rule_keeps_solid_at_melting_enthalpy():
    """Eq. 47: sigma_1 + sigma_4 = 2 keeps every node two cells ahead of the front at h_m."""
    w = inp.stefan_melting(enth_model=inp.ENTH_MRT, tau_g=1 / 1.14)
    err, _ = _solid_ahead_error(w, 3000)
    assert err <= 1e-13
    # case (c) of Sec. 3.1.2: sigma_4 = sigma_5 = 1.9 != 2 - sigma_1 leaks into the solid
    wc = inp.stefan_melting(enth_model=inp.ENTH_MRT, tau_g=1 / 1.14, sigma4=1.9)
    err_c, _ = _solid_ahead_error(wc, 3000)
    assert err_c > 1e-6


def test_srt_far_from_unit_tau_cools_the_solid():
    """Sec. 3.1.1: SRT with tau = 0.564 gives a solid temperature below T_m (the paper
    reports -0.00152 on its own grid); tau = 1 keeps the solid at T_m."""
    w = inp.stefan_melting(enth_model=inp.ENTH_SRT, tau_g=0.564)
    _, Tmin = _solid_ahead_error(w, 3000)
    assert Tmin < -1e-4
    w1 = inp.stefan_melting(enth_model=inp.ENTH_SRT, tau_g=1.0)
    err1, _ = _solid_ahead_error(w1, 3000)
    assert err1 <= 1e-13


def _melting_errors(enth_model, tau, steps, nx=96):
    """Front and temperature errors of Stefan melting (St = 0.1) against Eq. 60-61."""
    w = inp.stefan_melting(nx=nx, enth_model=enth_model, tau_g=tau)
    o = oracle.Oracle(w.shape, w.params)
    o.set_initial_h(inp.h0_field(w))
    o.step(steps)
    chi = o.lattice()["chi"]
    k = nm.melting_k(0.1)
    F = o.fields()
    T, fl = F["T"][0, 0, :], F["fl"][0, 0, :]
    x = np.arange(nx) + 0.5
    X = float(nm.melting_front(steps, chi, k))
    Ta = nm.melting_temperature(x, steps, chi, k)
    return (fl.sum() - X) / X, np.abs(T - Ta).max(), T[x > X + 2].min()


def test_srt_versus_mrt_over_the_relaxation_time():
    """Sec. 3.1.1 relaxation-time study (tau = 0.564, 1.012, 6.9): MRT follows Eq. 60-61 at
    every tau; SRT only near tau = 1 -- at 0.564 it cools the solid below T_m and lags, at
    6.9 it deviates at the interface."""
    for tau, steps in ((0.564, 20000), (1.012, 5000), (6.9, 1500)):
        ef_m, eT_m, Tmin_m = _melting_errors(inp.ENTH_MRT, tau, steps)
        ef_s, eT_s, Tmin_s = _melting_errors(inp.ENTH_SRT, tau, steps)
        assert abs(ef_m) < 5e-3 and abs(Tmin_m) < 1e-9
        if tau == 1.012:
            assert abs(ef_s) < 5e-3 and abs(Tmin_s) < 1e-6
        else:
            assert abs(ef_s) > 0.02
        if tau == 0.564:
            assert Tmin_s < -1e-3
        if tau == 6.9:
            assert eT_s > 0.1 and eT_m < 0.01


def _solidification_rule(sigma4, chi, t=20000, nx=96):
    w = inp.stefan_solidification(nx=nx, chi=chi)
    o = oracle.Oracle(w.shape, w.params.replace(sigma4=sigma4))
    o.set_initial_h(inp.h0_field(w))
    o.step(t)
    F = o.fields()
    T, fl = F["T"][0, 0, :], F["fl"][0, 0, :]
    k = nm.solidification_k(0.004, 0.004, chi, chi)
    x = np.arange(nx) + 0.5
    X = float(nm.solidification_front(t, chi, k))
    Ta = nm.solidification_temperature(x, t, chi, chi, k)
    liquid = (x > X + 1) & (x < X + 30)
    mushy = int(((fl > 1e-6) & (fl < 1 - 1e-6)).sum())
    return ((1 - fl).sum() - X) / X, np.abs(T[liquid] - Ta[liquid]).max(), mushy


def test_relaxation_rule_cases_c_and_d():
    """Sec. 3.1.2 cases (c)/(d): case (a) physics with sigma_1..3 = 1.14 and sigma_4..6 =
    2 - sigma_1 (Eq. 47), 1.9 (c) or 0.1 (d).  Breaking the rule moves the front and puts
    an error into the liquid ahead of it that the rule keeps out; (d) also widens the
    interface beyond one node."""
    chi = (1 / 1.14 - 0.5) * 0.25
    ef_r, eT_r, w_r = _solidification_rule(0.0, chi)
    ef_c, eT_c, w_c = _solidification_rule(1.9, chi)
    ef_d, eT_d, w_d = _solidification_rule(0.1, chi)
    assert abs(ef_r) < 0.02 and eT_r < 0.015 and w_r <= 1
    assert abs(ef_c) > 0.04 and eT_c > 3 * eT_r
    assert abs(ef_d) > 0.1 and eT_d > 3 * eT_r and w_d >= 3


def test_quasi_2d_convective_melting():
    """Sec. 3.2.2 (Table 1: Ra 2.5e4, Pr 0.02, Ste 0.01), 32 x 1 x 32: at Fo = 4 conduction
    dominates -- the melt depth equals the 1D Neumann value 2 k sqrt(Fo) (Eq. 61) and the
    interface is nearly vertical; by Fo = 10 convection bends it (more melt at the top, where
    the heated liquid rises) and melting runs ahead of pure conduction."""
    w = inp.cavity_melting_2d(n=32, precision=inp.FP64)
    o = oracle.Oracle(w.shape, w.params)
    o.set_initial_h(inp.h0_field(w))
    chi = o.lattice()["chi"]
    k = nm.melting_k(0.01)
    n, done = w.shape[0], 0
    for Fo in (4, 10):
        t = int(round(Fo * n * n / chi))
        o.step(t - done)
        done = t
        depth = o.fields()["fl"][:, 0, :].sum(axis=1) / n  # per z row, in cavity widths
        X = 2 * k * math.sqrt(Fo)
        if Fo == 4:
            assert abs(depth.mean() - X) / X < 0.01 and depth[-1] - depth[0] < 0.03
        else:
            assert depth.mean() > X and depth[-1] - depth[0] > 0.05


def test_corner_solidification():
    """Sec. 3.2.1 set-up (comparison data not in the container, so checked against what must
    hold): the field is symmetric about the diagonal; far from the corner the front and the
    temperature follow the 1D Neumann solution of Eq. 62-63 (Ste_s = 4, Ste_l = 1.2, equal
    chi); the corner, cooled from two sides, freezes further, by a depth ratio that stays
    constant in time (the problem is self-similar)."""
    w = inp.corner_solidification(n=128)
    o = oracle.Oracle(w.shape, w.params)
    o.set_initial_h(inp.h0_field(w))
    chi = 0.1
    k = nm.solidification_k(4.0, 1.2, chi, chi)
    x = np.arange(w.shape[0]) + 0.5
    ratios = []
    done = 0
    for t in (1125, 4500):
        o.step(t - done)
        done = t
        F = o.fields()
        fl, T = F["fl"][:, 0, :], F["T"][:, 0, :]  # (z, x)
        assert np.abs(T - T.T).max() < 1e-13
        X = float(nm.solidification_front(t, chi, k))
        far = (1.0 - fl[:, -1]).sum()  # depth along z at the far (mirror) column
        assert abs(far - X) <= max(0.03 * X, 0.6)
        Ta = nm.solidification_temperature(x, t, chi, chi, k, T0=0.3, T1=-1.0)
        assert np.abs(T[:, -1] - Ta).max() < 0.01
        ratios.append((1.0 - np.diag(fl)).sum() / X)
    assert ratios[0] > 1.1 and abs(ratios[1] / ratios[0] - 1) < 0.03


@pytest.mark.parametrize("enth_model", [inp.ENTH_SRT, inp.ENTH_MRT])
def test_steady_conduction_nusselt_is_one(enth_model):
    p = inp.Params(flow_model=0, enth_model=enth_model, tau_g=1.3,
                   bc=[inp.ISOTHERMAL, inp.ISOTHERMAL] + [inp.PERIODIC] * 4,
                   T_wall=[1.0, 0.0, 0, 0, 0, 0], St=1.0)
    o = oracle.Oracle((16, 1, 1), p)
    L = o.lattice()["latent"]
    o.set_initial_h(np.full(o.N, L + 0.5))
    o.step(12000)
    d = o.diagnostics()
    assert abs(d["nu_hot"] - 1.0) < 1e-9
    T = o.fields()["T"][0, 0, :]
    assert np.allclose(T, 1.0 - (np.arange(16) + 0.5) / 16, atol=1e-9)
