"""Host-side checks of the C ABI (no GPU needed).

The CUDA library must build here (nvcc cross-compiles sm_103a), load, export every
symbol include/lbpc.h declares, agree with the binding on the parameter-block
layout, size the workspace as documented, reject invalid inputs before any CUDA call,
and map the physical groups to the same lattice constants as the oracle does
independently (Eq. 20, 34, 52, 59, 64).
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import lbpc_inputs as inp
import oracle
from paper_1703_02652_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "lbpc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbpc_[a-z_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    L = B.lib()
    declared = _header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == declared


def test_param_block_layout_matches():
    L = B.lib()
    assert L.lbpc_params_size() == C.sizeof(B.LbpcParams)
    assert L.lbpc_abi_version() == 3


@pytest.mark.parametrize("precision,streaming,flow,per_node", [
    (inp.FP32, inp.PULL, inp.FLOW_MRT, 2 * 25 * 4 + 16),
    (inp.FP32, inp.AA, inp.FLOW_MRT, 25 * 4 + 16),
    (inp.FP16, inp.PULL, inp.FLOW_MRT, 2 * 25 * 2 + 16),
    (inp.BF16, inp.AA, inp.FLOW_MRT, 25 * 2 + 16),
    (inp.FP64, inp.PULL, inp.FLOW_NONE, 2 * 6 * 8 + 16),
    (inp.FP16_G32, inp.PULL, inp.FLOW_MRT, 2 * (19 * 2 + 6 * 4) + 16),
    (inp.BF16_G32, inp.AA, inp.FLOW_MRT, 19 * 2 + 6 * 4 + 16),
])
def test_workspace_bytes_per_node(precision, streaming, flow, per_node):
    p = inp.Params(precision=precision, streaming=streaming, flow_model=flow, tau_g=0.8)
    n = 128
    ws = B.workspace_bytes((n, n, n), p)
    ws_half = B.workspace_bytes((n // 2, n // 2, n // 2), p)
    assert ws >= per_node * n ** 3
    # the remainder (face fields, reduction scratch, history) grows at most with the area
    slope = (ws - ws_half) / (n ** 3 - (n // 2) ** 3)
    assert abs(slope - per_node) / per_node < 0.01


@pytest.mark.parametrize("bad", [
    dict(flow_model=7), dict(enth_model=0), dict(precision=6), dict(streaming=3),
    dict(bc=[0, 1, 2, 2, 2, 2]), dict(St=0.0), dict(omega_T=0.5), dict(Cp_s=-1.0),
    dict(Th=0.0), dict(tau_g=0.4), dict(Ra=-1.0), dict(Ma=2.0), dict(s_e=2.5),
    dict(sigma4=2.2), dict(report_every=-1),
])
def test_invalid_parameters_rejected_before_any_cuda_call(bad):
    p = inp.Params(**bad)
    L = B.lib()
    cp = B.to_c(p)
    assert L.lbpc_workspace_bytes(8, 8, 8, C.byref(cp)) == 0
    h = C.c_void_p()
    st = L.lbpc_create(8, 8, 8, C.byref(cp), None, 0, None, C.byref(h))
    assert st == B.LBPC_ERR_PARAM
    assert not h.value
    assert L.lbpc_last_error(None).decode()


def test_bad_extents_and_missing_workspace():
    L = B.lib()
    cp = B.to_c(inp.Params())
    h = C.c_void_p()
    assert L.lbpc_create(0, 8, 8, C.byref(cp), None, 0, None, C.byref(h)) == B.LBPC_ERR_PARAM
    assert L.lbpc_create(2048, 2048, 1024, C.byref(cp), None, 0, None,
                         C.byref(h)) == B.LBPC_ERR_PARAM
    # grid limits: ny and nz at most 65535 (the node count alone would be fine)
    assert L.lbpc_workspace_bytes(2, 2, 65536, C.byref(cp)) == 0
    assert L.lbpc_workspace_bytes(2, 65536, 2, C.byref(cp)) == 0
    assert L.lbpc_workspace_bytes(2, 2, 65535, C.byref(cp)) > 0
    st = L.lbpc_create(8, 8, 8, C.byref(cp), None, 0, None, C.byref(h))
    assert st == B.LBPC_ERR_WORKSPACE
    st = L.lbpc_create(8, 8, 8, C.byref(cp), C.c_void_p(256), 16, None, C.byref(h))
    assert st == B.LBPC_ERR_WORKSPACE
    st = L.lbpc_create(8, 8, 8, C.byref(cp), C.c_void_p(4096 + 8), 1 << 30, None, C.byref(h))
    assert st == B.LBPC_ERR_WORKSPACE  # misaligned


@pytest.mark.parametrize("shape,kw", [
    ((64, 64, 64), dict(Ra=1e5, Pr=0.02, St=1.0)),
    ((256, 256, 256), dict(Ra=1e6, Pr=50.0, St=1.0)),
    ((96, 96, 96), dict(Ra=1e5, Pr=6.2, St=1.0, flow_model=inp.FLOW_SRT)),
    ((64, 4, 4), dict(flow_model=inp.FLOW_NONE, tau_g=0.8, St=0.1)),
    ((40, 8, 8), dict(enth_model=inp.ENTH_SRT, Ra=1e4, Pr=1.0, St=0.3, sigma4=0.0)),
    ((40, 8, 8), dict(Ra=1e4, Pr=1.0, St=0.3, sigma4=1.5, s_e=1.1, s_q=1.3, Cp_l=2.0)),
])
def test_lattice_mapping_agrees_with_oracle(shape, kw):
    p = inp.Params(**kw)
    lib_l = B.lattice_constants(shape, p)
    orc = oracle.Oracle(shape, p, alloc=False).lattice()
    for k in ("chi", "nu", "gbeta", "sigma_chi", "sigma4", "s_nu", "latent", "hs", "hl",
              "tau_g", "tau_f", "s_e", "s_eps", "s_q", "s_pi", "s_t", "U0"):
        assert np.isclose(lib_l[k], orc[k], rtol=1e-14, atol=1e-300), k


def test_mapping_values_for_the_64_cube():
    lat = B.lattice_constants((64, 64, 64), inp.Params(Ra=1e5, Pr=0.02, St=1.0))
    assert np.isclose(lat["nu"], 0.1 / np.sqrt(3) * 64 * np.sqrt(0.02 / 1e5))
    assert np.isclose(lat["chi"], lat["nu"] / 0.02)
    assert np.isclose(lat["sigma_chi"] + lat["sigma4"], 2.0)  # Eq. 47
    assert np.isclose((1 / lat["s_nu"] - 0.5) / 3, lat["nu"])  # Eq. 59
    assert np.isclose((1 / lat["sigma_chi"] - 0.5) * 0.25, lat["chi"])  # Eq. 34
