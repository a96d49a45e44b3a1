"""Populations that cross isothermal walls keep FP32 precision in 16-bit g storage.

The wall flux of Eq. 65 is the difference of the population entering through an
isothermal wall (anti-bounce-back, -g*_out + omega_T C_p,ref T_w) and the one leaving, a
small difference of two O(0.1) values.  With g stored in 16 bits the leaving population
is kept as its 16-bit value plus an FP32 residual (per face, per boundary node), so the
entering one is formed from the FP32 value.  After each step from a random state (the
oracle continues from the GPU's state each step), the populations entering through the
isothermal x walls must therefore equal the oracle's to FP32 collision rounding (1e-6),
where the rest only meet one 16-bit ulp; with the 16-bit value alone they would be off by
up to half an FP16 ulp of 0.25 (6e-5) or a BF16 one (5e-4).  Pull and AA streaming (both
layouts), one node per thread (odd n_x) and node pairs (even n_x), a per-node wall field.
"""
import numpy as np
import pytest
import torch

import lbpc_inputs as inp
import oracle
from paper_1703_02652_gb300 import LBPC

pytestmark = pytest.mark.gpu

TOL16 = {inp.FP16: 2.5e-4, inp.BF16: 2e-3}


@pytest.mark.parametrize("precision", [inp.FP16, inp.BF16])
@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
@pytest.mark.parametrize("flow_model", [inp.FLOW_MRT, inp.FLOW_NONE])
@pytest.mark.parametrize("nx", [19, 20])
def test_wall_populations_keep_fp32_precision(precision, streaming, flow_model, nx):
    shape = (nx, 6, 5)
    p = inp.Params(flow_model=flow_model, precision=precision, streaming=streaming, Ra=5e4,
                   Pr=0.5, St=0.7, tau_g=0.0 if flow_model else 0.9,
                   bc=[inp.ISOTHERMAL, inp.ISOTHERMAL, inp.PERIODIC, inp.PERIODIC,
                       inp.ADIABATIC, inp.ADIABATIC], T_wall=[1.0, 0.0, 0, 0, 0, 0])
    Tw = inp.wall_temperature_field(6, 5, seed=3)
    f, gq = inp.random_state(shape, seed=9, flow=flow_model != 0)
    dev = torch.device("cuda")
    g = LBPC(shape, p)
    g.set_wall_temperature(0, Tw)
    g.set_distributions(torch.from_numpy(f).to(dev) if f is not None else None,
                        torch.from_numpy(gq).to(dev))
    o = oracle.Oracle(shape, p)
    o.set_wall_temperature(0, Tw)
    wall = np.zeros((7, 5, 6, nx), dtype=bool)  # populations entering through x walls
    wall[1, :, :, 0] = True
    wall[2, :, :, nx - 1] = True
    wall = wall.reshape(7, -1)
    for _ in range(3):
        f0, g0 = g.distributions()
        o.set_distributions(f0.cpu().numpy() if f0 is not None else None, g0.cpu().numpy())
        g.step(1)
        o.step(1)
        _, g1 = g.distributions()
        _, go = o.distributions()
        err = np.abs(g1.cpu().numpy() - go)
        assert err[wall].max() <= 1e-6, err[wall].max()
        assert err[1:].max() <= TOL16[precision]
