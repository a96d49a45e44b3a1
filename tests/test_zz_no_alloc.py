"""lbpc_get_scalars_noalloc: diagnostics without any device allocation.

The entry point serves callers that cannot allocate device memory when they read the
diagnostics (free memory owned by a pool, no cudaMalloc/cudaFree allowed because they
may synchronise the device, a fixed memory budget).  Its scratch is a static device
array inside the library.  Checked here through the C ABI against lbpc_get_scalars,
on two calls in a row, within the FP64 tolerance of the other diagnostics tests.
This file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import lbpc_inputs as inp
from paper_1703_02652_gb300 import LBPC
from paper_1703_02652_gb300 import binding as B

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _noalloc(lat, out):
    return B.lib().lbpc_get_scalars_noalloc(lat._h, C.c_void_p(out.data_ptr()))


def _check(got, ref):
    for i, k in enumerate(B.S_NAMES):
        assert abs(got[i] - ref[k]) <= RTOL * max(1.0, abs(ref[k])), (k, got[i], ref[k])


@pytest.mark.parametrize("streaming", [inp.PULL, inp.AA])
def test_noalloc_scalars_match_two_calls_in_a_row(streaming):
    shape = (24, 16, 12)
    p = inp.Params(precision=inp.FP32, streaming=streaming, Ra=1e5, Pr=0.71, St=1.0)
    lat = LBPC(shape, p)
    lat.set_initial_h(np.random.default_rng(0).uniform(-0.2, 1.5, int(np.prod(shape))))
    lat.step(51)
    out = torch.full((len(B.S_NAMES),), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row on the same state
        assert _noalloc(lat, out) == B.LBPC_OK
        _check(out.cpu().numpy(), lat.scalars())
    lat.step(31)  # and again after the state moved on, at an even step count (AA: the
    for _ in range(2):  # natural layout; above, after 51 steps, the swapped one)
        launches = lat.launch_count
        assert _noalloc(lat, out) == B.LBPC_OK
        assert lat.launch_count == launches + 2  # reduction pass and finalize
        _check(out.cpu().numpy(), lat.scalars())


def test_noalloc_rejects_oversized_lattice_and_null_output():
    out = torch.empty(len(B.S_NAMES), dtype=torch.float64, device="cuda")
    wide = LBPC((4097, 1, 1), inp.Params(precision=inp.FP32, flow_model=0, tau_g=0.9,
                                         bc=[inp.PERIODIC] * 6))
    assert _noalloc(wide, out) == B.LBPC_ERR_PARAM
    assert b"LBPC_NOALLOC_MAX_NX" in B.lib().lbpc_last_error(wide._h)
    small = LBPC((8, 8, 8), inp.Params(precision=inp.FP32))
    assert B.lib().lbpc_get_scalars_noalloc(small._h, None) == B.LBPC_ERR_PARAM
