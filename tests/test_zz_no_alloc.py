"""pfc_residual_static: the residual entry point for callers that cannot
allocate device memory (it takes no workspace and keeps its scratch in a fixed
array inside the library).  Checked against pfc_residual, the workspace-based
entry point, on two calls in a row, through the C ABI.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test has run in the same process."""
import ctypes
import math

import numpy as np
import pytest

from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H = math.pi / 4
GAMMA = 0.25


@pytest.fixture(scope="module")
def pfc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P


def static_residual(P, torch, shape, Phi, phin, dt):
    F = torch.empty(shape, dtype=torch.float64, device="cuda")
    nrm = ctypes.c_double(-1.0)
    st = torch.cuda.current_stream()
    rc = P.lib().pfc_residual_static(ctypes.byref(P.make_grid(shape)), H, GAMMA, ctypes.c_void_p(Phi.data_ptr()),
                                     ctypes.c_void_p(phin.data_ptr()), dt, ctypes.c_void_p(F.data_ptr()),
                                     ctypes.byref(nrm), ctypes.c_void_p(st.cuda_stream))
    assert rc == P.PFC_OK, P.status_str(rc)
    return F, nrm.value


@pytest.mark.parametrize("shape", [(64, 64), (40, 70)])
def test_static_residual_matches_workspace_residual_twice(pfc, shape):
    import torch

    s = pfc.Solver(shape, H, GAMMA, pfc.default_params(sub=(1, 1), overlap=0))
    for call, (seed, dt) in enumerate([(1, 0.7), (2, 9.0)]):  # two calls in a row, different data
        Phi = torch.from_numpy(inputs.noise_field(shape, 0.2, 0.4, 10 * seed)).cuda()
        phin = torch.from_numpy(inputs.noise_field(shape, 0.2, 0.4, 10 * seed + 1)).cuda()
        F_ref, n_ref = s.residual(Phi, phin, dt)
        F, n = static_residual(pfc, torch, shape, Phi, phin, dt)
        ref = F_ref.cpu().numpy()
        np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert n == pytest.approx(n_ref, rel=1e-12), call


def test_static_residual_rejects_oversized_grid(pfc):
    import torch

    # 8192 x 8192 cells = 131,072 tiles of 32 x 16: beyond the fixed scratch
    g = pfc.make_grid((8192, 8192))
    dummy = torch.empty(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = pfc.lib().pfc_residual_static(ctypes.byref(g), H, GAMMA, p, p, 1.0, p, None, None)
    assert rc == pfc.PFC_EINVAL
