"""Failure detection without a GPU fault.

* The bounded device-side wait that guards every mbarrier wait of the TMA copy
  rings: a one-CTA kernel waits on a barrier whose phase never completes (no
  arrival, no copy in flight) with a short cycle limit; it must give up, report
  PFC_ETIMEOUT through the C ABI and leave the context usable.
* Failed steps are transactional (the boundary's contract): a NaN planted on
  the host in a caller-supplied Newton guess makes pfc_step return PFC_ENAN,
  and a GMRES iteration cap makes it return PFC_EGMRES; in both cases phi^n,
  phi^{n-1} and the adaptive-step history are unchanged, compared byte for byte
  through the checkpoint files pfc_save writes before and after."""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H = math.pi / 4
GAMMA = 0.25


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P, torch


def test_bounded_wait_runs_out_and_reports_timeout(env):
    P, torch = env
    st = torch.cuda.Stream()
    flag = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    ptr, sp = ctypes.c_void_p(flag.data_ptr()), ctypes.c_void_p(st.cuda_stream)
    # no arrival: the phase never completes and the wait gives up after ~1e6 cycles (~0.5 ms)
    assert P.lib().pfc_wait_selftest(0, 1_000_000, ptr, sp) == P.PFC_ETIMEOUT
    assert int(flag.item()) == P.PFC_ETIMEOUT
    # one arrival completes the phase: the same wait succeeds
    assert P.lib().pfc_wait_selftest(1, 1_000_000, ptr, sp) == P.PFC_OK
    assert int(flag.item()) == P.PFC_OK
    # the context is still usable: a residual through the ordinary path matches the oracle
    shape = (32, 48)
    s = P.Solver(shape, H, GAMMA, P.default_params(sub=(2, 2)))
    Phi = inputs.noise_field(shape, 0.1, 0.3, 3)
    F, nrm = s.residual(Phi, Phi, 1.0)
    assert nrm == pytest.approx(np.linalg.norm(O.residual(Phi, Phi, 1.0, H, GAMMA)), rel=1e-12)
    s.close()


def _state_bytes(s, tmp_path, tag):
    path = os.path.join(str(tmp_path), f"ckpt_{tag}.bin")
    s.save(path)
    with open(path, "rb") as f:
        return f.read()


def _two_steps(P, params, shape=(48, 48)):
    s = P.Solver(shape, H, GAMMA, params)
    s.set_field(inputs.noise_field(shape, 0.07, 0.07, 1040))
    s.run(2)  # phi^n != phi^{n-1} and an energy history exist
    return s


def test_nan_guess_fails_cleanly_and_leaves_the_state(env, tmp_path):
    P, torch = env
    params = P.default_params(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0, guess=P.PFC_GUESS_USER)
    s = _two_steps(P, params)
    before = _state_bytes(s, tmp_path, "a")
    dt0 = s.next_dt()
    bad = s.get_field()
    bad[7, 11] = np.nan  # planted on the host
    s.set_guess(bad)
    with pytest.raises(P.PfcError) as e:
        s.step(dt0)
    assert e.value.status == P.PFC_ENAN
    assert _state_bytes(s, tmp_path, "b") == before
    assert s.next_dt() == dt0
    # the state still steps: without a guess Newton starts from phi^n and converges
    s.step(dt0)
    s.close()


def test_gmres_cap_fails_cleanly_and_leaves_the_state(env, tmp_path):
    P, torch = env
    params = P.default_params(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0, gmres_max_it=4)
    s = _two_steps(P, P.default_params(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0))
    path = os.path.join(str(tmp_path), "ckpt_src.bin")
    s.save(path)
    s.close()
    capped = P.Solver((48, 48), H, GAMMA, params)
    capped.load(path)
    before = _state_bytes(capped, tmp_path, "c")
    with pytest.raises(P.PfcError) as e:
        capped.step(10.0)
    assert e.value.status == P.PFC_EGMRES
    assert _state_bytes(capped, tmp_path, "d") == before
    capped.close()
