"""Pins of the oracle's reference adjoint.

* The complex-step node Jacobian equals central finite differences of the real
  node collision of the oracle (every inversion branch, with and without flow).
* The full adjoint's dJ/dT_w and dJ/dSt equal central finite differences of
  J = sum f_l(h_N) computed by the oracle's forward run (initial state held fixed,
  as the adjoint defines it).
* Dot-product consistency: dJ/dT_w . v equals the directional finite difference.
* All of it also with the enthalpy-porosity solid drag in place of the liquid-fraction
  closure.
"""
import numpy as np
import pytest

import lbpc_inputs as inp
import oracle


def _rand_node(o, rng, h, flow):
    f = (1 / 19) * (1 + 0.2 * rng.uniform(-1, 1, 19)) if flow else None
    g = np.concatenate([[0.0], rng.uniform(0.05, 0.2, 6)])
    g[0] = h - g[1:].sum()
    return f, g


@pytest.mark.parametrize("flow_model,enth_model,darcy_A", [(1, 1, 0.0), (2, 2, 0.0), (0, 1, 0.0),
                                                          (0, 2, 0.0), (1, 1, 5.0)])
@pytest.mark.parametrize("branch", ["solid", "mushy", "liquid"])
def test_complex_step_jacobian_matches_finite_differences(flow_model, enth_model, darcy_A,
                                                          branch):
    p = inp.Params(flow_model=flow_model, enth_model=enth_model, Ra=3e4, Pr=0.7, St=0.8,
                   tau_g=0.0 if flow_model else 0.9, Cp_l=1.3, darcy_A=darcy_A)
    o = oracle.Oracle((1, 1, 1), p, alloc=False)
    L = o.lattice()["latent"]
    h = {"solid": -0.3, "mushy": 0.4 * L, "liquid": L + 0.5}[branch]
    rng = np.random.default_rng(0)
    f, g = _rand_node(o, rng, h, flow_model != 0)
    J, dL = o.collide_jacobian(f, g)
    flow = flow_model != 0
    n = 26 if flow else 7
    x0 = np.concatenate([f, g]) if flow else g.copy()

    def F(x, Lshift=0.0):
        fp, gp, _ = o.collide_node(x[:19] if flow else None, x[19:] if flow else x)
        return np.concatenate([fp, gp]) if flow else gp

    eps = 1e-6
    Jfd = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = eps
        Jfd[:, i] = (F(x0 + e) - F(x0 - e)) / (2 * eps)
    assert np.abs(J - Jfd).max() <= 1e-8
    # dC/dL: perturb St, which moves L = C_p,l dT / St
    St = 0.8
    dSt = 1e-7
    outs = []
    for s in (St + dSt, St - dSt):
        o2 = oracle.Oracle((1, 1, 1), p.replace(St=s), alloc=False)
        fp, gp, _ = o2.collide_node(f, g)
        outs.append(np.concatenate([fp, gp]) if flow else gp)
    dLdSt = -1.3 * 1.0 / St ** 2
    assert np.abs((outs[0] - outs[1]) / (2 * dSt) - dL * dLdSt).max() <= 1e-6


def _cavity(flow_model=1, enth_model=1, darcy_A=0.0):
    shape = (6, 5, 4)
    p = inp.Params(flow_model=flow_model, enth_model=enth_model, precision=inp.FP64, Ra=2e4,
                   Pr=0.7, St=0.8, tau_g=0.0 if flow_model else 0.9, darcy_A=darcy_A)
    h0 = np.random.default_rng(3).uniform(-0.3, 1.6, int(np.prod(shape)))
    Tw = inp.wall_temperature_field(shape[1], shape[2], seed=1)
    o = oracle.Oracle(shape, p)
    o.set_wall_temperature(0, Tw)
    o.set_initial_h(h0)
    f0, g0 = o.distributions()
    return shape, p, Tw, f0, g0


def _J(shape, p, Tw, f0, g0, steps):
    o = oracle.Oracle(shape, p)
    o.set_wall_temperature(0, Tw)
    o.set_distributions(f0, g0)
    o.step(steps)
    return o.fields()["fl"].sum()


@pytest.mark.parametrize("flow_model,enth_model,darcy_A", [(1, 1, 0.0), (2, 2, 0.0), (0, 1, 0.0),
                                                          (1, 1, 5.0)])
def test_adjoint_gradients_match_finite_differences(flow_model, enth_model, darcy_A):
    shape, p, Tw, f0, g0 = _cavity(flow_model, enth_model, darcy_A)
    steps = 25
    o = oracle.Oracle(shape, p)
    o.set_wall_temperature(0, Tw)
    o.set_distributions(f0, g0)
    J, dTw, dSt = o.adjoint(steps, face=0)
    assert abs(J - _J(shape, p, Tw, f0, g0, steps)) <= 1e-12 * abs(J)
    eps = 1e-5
    for i in (0, 7, 13, 19):
        T1, T2 = Tw.copy(), Tw.copy()
        T1[i] += eps
        T2[i] -= eps
        fd = (_J(shape, p, T1, f0, g0, steps) - _J(shape, p, T2, f0, g0, steps)) / (2 * eps)
        assert abs(dTw[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, dTw[i], fd)
    e = 1e-6
    fd = (_J(shape, p.replace(St=p.St + e), Tw, f0, g0, steps)
          - _J(shape, p.replace(St=p.St - e), Tw, f0, g0, steps)) / (2 * e)
    assert abs(dSt - fd) <= 1e-6 * max(1.0, abs(fd)), (dSt, fd)
    # directional derivative along a random wall perturbation
    v = np.random.default_rng(9).standard_normal(Tw.size)
    fd = (_J(shape, p, Tw + 1e-6 * v, f0, g0, steps)
          - _J(shape, p, Tw - 1e-6 * v, f0, g0, steps)) / 2e-6
    assert abs(dTw @ v - fd) <= 1e-6 * max(1.0, abs(fd))
