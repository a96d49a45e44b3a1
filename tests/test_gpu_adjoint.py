"""GPU adjoint (reverse mode of the coupled step, through the C ABI).

* FP64 mode equals the oracle's reference adjoint (complex-step node Jacobians,
  transposed stream) on tiny lattices for every model combination.
* The checkpoint interval changes the result only at float rounding of the trajectory
  (the plain and the taping step are separate instantiations of one kernel).
* FP32 gradients agree with FP64 gradients.
* The torch.autograd.Function returns the same gradients.
* The 96^3 adjoint workload (Ra 1e5, Pr 6.2, St 1, hot-wall field 1 + 0.05 N(0,1),
  2000 steps, checkpoints every 100): central finite differences with eps = 1e-4 at 16
  seeded wall nodes and in St, forward in FP64 (FP32 rounding of the forward would
  swamp differences of ~1e-4), relative agreement 1e-4.
"""
import numpy as np
import pytest
import torch

import lbpc_inputs as inp
import oracle
from paper_1703_02652_gb300 import LBPC, LbpcError, liquid_volume
from paper_1703_02652_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _tiny(flow_model, enth_model, precision=inp.FP64):
    shape = (6, 5, 4)
    p = inp.Params(flow_model=flow_model, enth_model=enth_model, precision=precision, Ra=2e4,
                   Pr=0.7, St=0.8, tau_g=0.0 if flow_model else 0.9)
    h0 = np.random.default_rng(3).uniform(-0.3, 1.6, int(np.prod(shape)))
    Tw = inp.wall_temperature_field(shape[1], shape[2], seed=1)
    return shape, p, h0, Tw


@pytest.mark.parametrize("flow_model,enth_model,darcy_A", [
    (1, 1, 0.0), (2, 2, 0.0), (1, 2, 0.0), (0, 1, 0.0), (0, 2, 0.0), (1, 1, 5.0)])
def test_adjoint_equals_oracle_adjoint(flow_model, enth_model, darcy_A):
    shape, p, h0, Tw = _tiny(flow_model, enth_model)
    p = p.replace(darcy_A=darcy_A)
    g = LBPC(shape, p)
    g.set_wall_temperature(0, Tw)
    g.set_initial_h(h0)
    J, dTw, dSt = g.adjoint(25, 7, face=0)
    o = oracle.Oracle(shape, p)
    o.set_wall_temperature(0, Tw)
    o.set_initial_h(h0)
    Jo, dTwo, dSto = o.adjoint(25, face=0)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert np.abs(dTw - dTwo).max() <= 1e-10 * np.abs(dTwo).max()
    assert abs(dSt - dSto) <= 1e-10 * abs(dSto)
    assert g.step_count == 25  # left at the final state


def test_adjoint_other_face_and_walls():
    """Gradient with respect to the temperature of the +z face (isothermal there)."""
    shape = (5, 6, 7)
    p = inp.Params(flow_model=1, precision=inp.FP64, Ra=2e4, Pr=0.7, St=0.8,
                   bc=[inp.ISOTHERMAL, inp.ADIABATIC, inp.PERIODIC, inp.PERIODIC, inp.ADIABATIC,
                       inp.ISOTHERMAL], T_wall=[1.0, 0, 0, 0, 0, 0.3])
    h0 = np.random.default_rng(4).uniform(-0.3, 1.6, int(np.prod(shape)))
    g = LBPC(shape, p)
    g.set_initial_h(h0)
    J, dTw, dSt = g.adjoint(20, 6, face=5)
    o = oracle.Oracle(shape, p)
    o.set_initial_h(h0)
    Jo, dTwo, dSto = o.adjoint(20, face=5)
    assert np.abs(dTw - dTwo).max() <= 1e-10 * np.abs(dTwo).max()
    assert abs(dSt - dSto) <= 1e-10 * abs(dSto)


def test_checkpoint_interval_does_not_change_the_gradient():
    shape, p, h0, Tw = _tiny(1, 1, inp.FP32)
    res = []
    for k in (1, 5, 30):
        g = LBPC(shape, p)
        g.set_wall_temperature(0, Tw)
        g.set_initial_h(h0)
        res.append(g.adjoint(30, k))
    # The taping step is its own instantiation of the step kernel (the forward tapes its last
    # segment), so its FMA contraction may differ from the plain step's in the last bit of
    # a float: J agrees to float rounding of the trajectory, the gradients (FP32 adjoint
    # populations) to a few float ulps.
    for J, dTw, dSt in res[1:]:
        assert abs(J - res[0][0]) <= 1e-8 * abs(res[0][0])
        assert abs(dSt - res[0][2]) <= 1e-6 * abs(res[0][2])
        assert np.abs(dTw - res[0][1]).max() <= 1e-6 * np.abs(res[0][1]).max()


def test_fp32_gradients_track_fp64():
    shape = (20, 12, 10)
    res = {}
    for prec in (inp.FP64, inp.FP32):
        p = inp.Params(precision=prec, Ra=1e5, Pr=6.2, St=1.0)
        g = LBPC(shape, p)
        g.set_wall_temperature(0, inp.wall_temperature_field(12, 10, seed=0))
        g.set_initial_h(inp.h0_field(inp.cavity_melting(shape=shape)))
        res[prec] = g.adjoint(300, 50)
    J64, g64, s64 = res[inp.FP64]
    J32, g32, s32 = res[inp.FP32]
    assert abs(J32 - J64) <= 1e-5 * abs(J64)
    assert np.abs(g32 - g64).max() <= 1e-3 * np.abs(g64).max()
    assert abs(s32 - s64) <= 1e-3 * abs(s64)


@pytest.mark.parametrize("precision", [inp.FP32, inp.FP16])
def test_paired_tape_path(precision):
    """A lattice wide enough (even nx, whole warps of interior rows) that the forward tail,
    the segment recomputations and the plain steps run the two-nodes-per-thread kernels:
    the gradient does not depend on the checkpoint interval, and tracks FP64."""
    shape = (64, 8, 6)
    ny, nz = shape[1], shape[2]
    h0 = inp.h0_field(inp.cavity_melting(shape=shape))
    Tw = inp.wall_temperature_field(ny, nz, seed=2)
    res = {}
    for prec, k in ((precision, 1), (precision, 8), (precision, 40), (inp.FP64, 40)):
        p = inp.Params(precision=prec, Ra=1e5, Pr=6.2, St=1.0)
        g = LBPC(shape, p)
        g.set_wall_temperature(0, Tw)
        g.set_initial_h(h0)
        g.step(60)  # some melt first, so that the gradient is not zero
        res[(prec, k)] = g.adjoint(40, k)
    J1, g1, s1 = res[(precision, 1)]
    for k in (8, 40):
        J, gk, sk = res[(precision, k)]
        # the forward tail runs the taping instantiation of the step kernel, whose FP32
        # contraction may differ from the plain step's by an ulp here and there
        assert abs(J - J1) <= 1e-7 * abs(J1)
        assert np.abs(gk - g1).max() <= 1e-6 * np.abs(g1).max()
        assert abs(sk - s1) <= 1e-6 * abs(s1)
    J64, g64, s64 = res[(inp.FP64, 40)]
    tol = 1e-3 if precision == inp.FP32 else 5e-2
    print(precision, abs(J1 / J64 - 1), np.abs(g1 - g64).max() / np.abs(g64).max(), abs(s1 / s64 - 1))
    assert abs(J1 - J64) <= (1e-4 if precision == inp.FP32 else 1e-3) * abs(J64)
    assert np.abs(g1 - g64).max() <= tol * np.abs(g64).max()
    assert abs(s1 - s64) <= tol * abs(s64)


def test_autograd_function_matches_adjoint():
    shape, p, h0, Tw = _tiny(1, 1)
    T = torch.tensor(Tw, dtype=torch.float64, requires_grad=True)
    St = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    J = liquid_volume(T, St, shape, p, h0, 25, 7)
    (2.0 * J).backward()
    g = LBPC(shape, p)
    g.set_wall_temperature(0, Tw)
    g.set_initial_h(h0)
    Jr, dTw, dSt = g.adjoint(25, 7)
    assert abs(J.item() - Jr) <= 1e-12 * Jr
    assert np.allclose(T.grad.numpy(), 2.0 * dTw, rtol=1e-12, atol=0)
    assert abs(St.grad.item() - 2.0 * dSt) <= 1e-12 * abs(dSt)


def test_adjoint_error_paths():
    shape, p, h0, Tw = _tiny(1, 1)
    g = LBPC(shape, p.replace(streaming=inp.AA))
    with pytest.raises(LbpcError) as e:
        g.adjoint(5, 2)
    assert e.value.status == B.LBPC_ERR_STATE
    g = LBPC(shape, p)
    with pytest.raises(LbpcError) as e:
        g.adjoint_backward(0)
    assert e.value.status == B.LBPC_ERR_STATE
    g.adjoint_forward(5, 2)
    g.step(1)  # stepping in between invalidates the recorded trajectory
    with pytest.raises(LbpcError) as e:
        g.adjoint_backward(0)
    assert e.value.status == B.LBPC_ERR_STATE
    w = inp.stefan_solidification_b(nx=8, ny=3, nz=3)  # per-phase conductivities
    g = LBPC(w.shape, w.params)
    g.set_initial_h(inp.h0_field(w))
    with pytest.raises(LbpcError) as e:
        g.adjoint(5, 2)
    assert e.value.status == B.LBPC_ERR_STATE


def test_adjoint_workload_96_finite_differences():
    """Adjoint configuration: 96^3 cavity, Ra 1e5, Pr 6.2, St 1, T_w(y, z) = 1 + 0.05 N(0,1),
    2000 steps, checkpoints every 100; central differences with eps = 1e-4."""
    n, steps, k, eps = 96, 2000, 100, 1e-4
    w = inp.cavity_melting(n=n, Ra=1e5, Pr=6.2, St=1.0, precision=inp.FP64, report_every=0)
    p = w.params
    h0 = inp.h0_field(w)
    Tw = inp.wall_temperature_field(n, n, seed=0)
    nodes = inp.fd_wall_nodes(n, n, count=16, seed=0)

    lat = LBPC(w.shape, p)
    lat.set_wall_temperature(0, Tw)
    lat.set_initial_h(h0)
    J, dTw, dSt = lat.adjoint(steps, k)
    lat.release_adjoint_workspace()
    del lat
    torch.cuda.empty_cache()
    run = LBPC(w.shape, p)

    def J_of(Twf, St=1.0):
        if St != 1.0:
            r = LBPC(w.shape, p.replace(St=St))
        else:
            r = run
        r.set_wall_temperature(0, Twf)
        r.set_initial_h(h0)
        r.step(steps)
        return r.scalars()["liquid_vol"]

    assert abs(J_of(Tw) - J) <= 1e-12 * J
    errs = []
    for i in nodes:
        Tp, Tm_ = Tw.copy(), Tw.copy()
        Tp[i] += eps
        Tm_[i] -= eps
        fd = (J_of(Tp) - J_of(Tm_)) / (2 * eps)
        errs.append(abs(dTw[i] - fd) / max(abs(fd), 1e-300))
    assert max(errs) <= 1e-4, errs
    fd = (J_of(Tw, 1.0 + eps) - J_of(Tw, 1.0 - eps)) / (2 * eps)
    assert abs(dSt - fd) <= 1e-4 * abs(fd), (dSt, fd)
    # the FP32 forward's gradient against the FP64 one
    lat32 = LBPC(w.shape, p.replace(precision=inp.FP32))
    lat32.set_wall_temperature(0, Tw)
    lat32.set_initial_h(h0)
    J32, dTw32, dSt32 = lat32.adjoint(steps, k)
    assert abs(J32 - J) <= 1e-4 * J
    assert np.abs(dTw32 - dTw).max() <= 2e-2 * np.abs(dTw).max()
