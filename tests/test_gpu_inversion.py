"""The Eq. 2 inversion (h -> T, f_l) at its kinks, on the GPU, against the oracle.

The excess e = h - h_s is FP64 in every storage mode.  Fields and diagnostics report the
FP64 inversion of it; the FP32 collision of the 32/16-bit modes inverts e rounded once to
nearest.  Enthalpies placed a few FP64 ulps to 1e-6 away from h_s and h_l (and on them), and
fractions of an FP32 ulp of L above h_l, must therefore give:

* fields: T and f_l equal to the oracle's to FP64 rounding, 4e-15 absolute, in every
  storage mode, both kinks, unequal specific heats, a latent heat that is not a float;
* one step in 32-bit g storage: each moving population of a node that starts at the
  equilibrium of its own temperature is (omega_T / 2) C_p,ref T of its upwind node after
  the step, so its error is at most that of T, half an FP32 ulp of e over C_p (plus FP32
  rounding).  Truncation instead of rounding to nearest errs by up to a whole ulp and
  fails at the offsets of 0.7 and 1.7 ulps.
"""
import numpy as np
import pytest
import torch

import lbpc_inputs as inp
import oracle
from paper_1703_02652_gb300 import LBPC

pytestmark = pytest.mark.gpu

DELTAS = np.array([0.0, 1e-15, 1e-12, 1e-9, 3e-8, 1e-7, 1e-6])
CASES = {  # T_m, C_p,s, C_p,l, St (L = C_p,l (T_h - T_m) / St, T_h = 1)
    "Tm0": (0.0, 1.0, 2.0, 0.7),
    "Tm025": (0.25, 1.5, 0.75, 1.3),
}


def _kink_enthalpies(hs, hl, n_random, seed):
    d = np.concatenate([-DELTAS[::-1], DELTAS[1:]])
    rng = np.random.default_rng(seed)
    h = np.concatenate([hs + d, hl + d, rng.uniform(hs - 0.5, hl + 0.5, n_random)])
    return rng.permutation(h)


def _params(case, precision, streaming=inp.PULL):
    Tm, Cps, Cpl, St = CASES[case]
    return inp.Params(flow_model=inp.FLOW_NONE, enth_model=inp.ENTH_MRT, precision=precision,
                      streaming=streaming, bc=[inp.PERIODIC] * 6, tau_g=0.9, Tm=Tm, Th=1.0,
                      Tref=Tm, Cp_s=Cps, Cp_l=Cpl, Cp_ref=1.0, St=St)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [inp.FP64, inp.FP32, inp.FP16, inp.BF16, inp.FP16_G32,
                                       inp.BF16_G32])
def test_fields_at_the_kinks(case, precision):
    shape = (16, 4, 3)
    p = _params(case, precision)
    o = oracle.Oracle(shape, p)
    lat = o.lattice()
    h = _kink_enthalpies(lat["hs"], lat["hl"], int(np.prod(shape)) - 26, seed=1)
    g = LBPC(shape, p)
    g.set_initial_h(h)
    F = {k: v.cpu().numpy().ravel() for k, v in g.fields().items()}
    T_o = np.empty_like(h)
    fl_o = np.empty_like(h)
    for i, hv in enumerate(h):
        T_o[i], fl_o[i] = o.invert(hv)
    assert np.abs(F["h"] - h).max() <= 4e-15
    assert np.abs(F["T"] - T_o).max() <= 4e-15
    assert np.abs(F["fl"] - fl_o).max() <= 4e-15
    assert F["fl"].min() >= 0.0 and F["fl"].max() <= 1.0
    # every branch is present, with values within 1e-15 of both kinks
    assert (fl_o == 0).any() and (fl_o == 1).any() and ((fl_o > 0) & (fl_o < 1)).any()


@pytest.mark.parametrize("precision", [inp.FP32, inp.FP16_G32])
@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
@pytest.mark.parametrize("nx", [15, 16])  # one node per thread / node pairs
def test_step_inversion_at_the_kinks(precision, streaming, nx):
    shape = (nx, 4, 3)
    # C_p,l = 2, St = 0.5: L = 4 is a float, so the only rounding in T is that of e
    p = _params("Tm0", precision, streaming).replace(St=0.5)
    o = oracle.Oracle(shape, p)
    lat = o.lattice()
    hs, hl = lat["hs"], lat["hl"]
    assert hl == 4.0
    ulp_L = float(np.spacing(np.float32(hl)))
    N = int(np.prod(shape))
    rng = np.random.default_rng(2)
    near = hl + ulp_L * np.array([0.3, 0.7, 1.3, 1.7, -0.3, -0.7, -1.3])
    base = _kink_enthalpies(hs, hl, N - 26 - near.size, seed=2)
    h = rng.permutation(np.concatenate([base, near]))
    g = LBPC(shape, p)
    g.set_initial_h(h)
    _, g0 = g.distributions()
    o.set_distributions(None, g0.cpu().numpy())
    g.step(1)
    o.step(1)
    _, g1 = g.distributions()
    _, go = o.distributions()
    g1 = g1.cpu().numpy()
    # per node: half an FP32 ulp of its excess over its branch's C_p (0 in the mushy zone,
    # where T = T_m), carried to the downwind populations of the periodic box
    e = (h - hs).reshape(shape[::-1])
    cp = np.where(e <= 0, p.Cp_s, p.Cp_l)
    tolT = np.where((e > 0) & (e < hl - hs), 0.0,
                    0.5 * np.spacing(np.abs(e).astype(np.float32)).astype(np.float64) / cp)
    ex = [(1, 2), (-1, 2), (1, 1), (-1, 1), (1, 0), (-1, 0)]  # D3Q7 a = 1..6: shift, axis
    for a_, (sh, ax) in enumerate(ex, start=1):
        tol = 0.125 * np.roll(tolT, sh, axis=ax).ravel() * (1 + 1e-6)
        err = np.abs(g1[a_] - go[a_])
        # (1e-15: the oracle's own FP64 rounding, where both should be 0 at mushy nodes)
        bad = err > tol + 2.0 ** -22 * np.abs(go[a_]) + 1e-15
        assert not bad.any(), (a_, err[bad].max(), tol[bad].max())
    # the nodes near the liquid kink carry temperatures below one FP32 ulp of L
    assert ((np.abs(go[1:]) > 0) & (np.abs(go[1:]) < 1e-7)).sum() >= 6
