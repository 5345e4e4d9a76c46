"""GPU parity at the workloads' full sizes, in the configuration bench.py times
(1024^2 and 2048^2 with 64^2 / 128^2 cores of 16^2, BF16 factors, learned
guess; 256^3 with 7^3 uneven cores).  The oracle evaluates whole-grid
operators directly (residual, JVP, energy, mass: plain stencils), the Schwarz
apply on sampled subdomains (a core of the left-RAS output depends on its own
block only), and checks time steps through properties that hold at any size:
the oracle's residual of the GPU's phi^{n+1} meets the Newton tolerance, mass
is conserved and the discrete energy does not increase."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, learned, pfc as P

    build.build()
    P.lib()
    return P, torch, learned


def _solver(P, learned, w, prec, guess_learned=False, gamma=None):
    params = P.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                              dt_max=w["dt_max"], eta=w["eta"],
                              guess=P.PFC_GUESS_LEARNED if guess_learned else P.PFC_GUESS_PREV)
    s = P.Solver(w["shape"], w["h"], w["gamma"] if gamma is None else gamma, params)
    net = None
    if guess_learned:
        theta, s_out = learned.load()
        net = P.GuessNet(w["shape"])
        net.set_params(theta)
        P.set_guess_net(s, net, s_out)
    return s, net


@pytest.mark.parametrize("name", ["hex1024", "hex2048", "bcc256"])
def test_operators_at_full_size(env, name):
    """Residual, JVP, energy and mass over the whole grid against the oracle."""
    P, torch, learned = env
    w = inputs.workload(name)
    s, _ = _solver(P, learned, w, 1)
    phin = w["phi"]
    Phi = phin + inputs.noise_field(w["shape"], 0.0, 0.01, 77)
    v = inputs.noise_field(w["shape"], 0.0, 1.0, 78)
    dt = 10.0
    F, nrm = s.residual(Phi, phin, dt)
    ref = O.residual(Phi, phin, dt, w["h"], w["gamma"])
    assert np.abs(F.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    del F, ref
    Jv = s.jvp(Phi, phin, v, dt).cpu().numpy()
    ref = O.jvp(v, Phi, phin, dt, w["h"], w["gamma"])
    assert np.abs(Jv - ref).max() <= 1e-12 * np.abs(ref).max()
    del Jv, ref
    s.set_field(phin)
    assert s.energy() == pytest.approx(O.energy(phin, w["h"], w["gamma"]), rel=1e-12)
    assert s.mass() == pytest.approx(O.mass(phin, w["h"]), rel=1e-12)
    s.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (2, 0.25)])
def test_schwarz_apply_on_sampled_blocks_1024(env, prec, tol):
    """z = sum_k (R_k^0)^T A_k^{-1} R_k^delta r on the 4096-block 1024^2 case: the
    cores of 8 sampled blocks (corners with periodic wrap included) against dense
    solves with the oracle's improved-BC block matrices."""
    P, torch, learned = env
    w = inputs.workload("hex1024")
    s, _ = _solver(P, learned, w, prec)
    phin = w["phi"]
    Phi = phin + inputs.noise_field(w["shape"], 0.0, 0.01, 79)
    r = inputs.noise_field(w["shape"], 0.0, 1.0, 80)
    dt = 10.0
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy().ravel()
    blocks = O.decompose(w["shape"], w["parts"], 1)
    for k in (0, 63, 64, 2047, 2080, 4032, 4095, 1234):
        blk = blocks[k]
        A = O.subdomain_matrix_improved_bc(Phi, phin, dt, w["h"], w["gamma"], blk)
        sol = scipy.linalg.solve(A, r.ravel()[blk.block_idx])[blk.core_mask]
        got = z[blk.core_idx]
        assert np.linalg.norm(got - sol) / np.linalg.norm(sol) <= tol, k
    s.close()


@pytest.mark.parametrize("name,prec,learned_guess", [("hex1024", 2, True), ("hex1024", 0, False),
                                                     ("hex2048", 2, True), ("bcc256", 1, False)])
def test_time_steps_at_full_size_satisfy_the_scheme(env, name, prec, learned_guess):
    """Two adaptive steps (dt_min, then the controller's dt): the oracle's residual of
    each GPU phi^{n+1} is within the Newton tolerance 1e-10 ||F(phi^n)||, mass is
    conserved to 1e-12 and the energy does not increase (Eq. NSOP, Sec. 3)."""
    P, torch, learned = env
    w = inputs.workload(name)
    s, net = _solver(P, learned, w, prec, learned_guess and len(w["shape"]) == 2)
    s.set_field(w["phi"])
    prev = w["phi"]
    for _ in range(2):
        info = s.run(1)[0]
        cur = s.get_field()
        dt = info["dt"]
        r_new = np.linalg.norm(O.residual(cur, prev, dt, w["h"], w["gamma"]))
        r_ref = np.linalg.norm(O.residual(prev, prev, dt, w["h"], w["gamma"]))
        assert r_new <= 1e-10 * r_ref * 1.01 + 1e-13 * math.sqrt(prev.size)
        m0, m1 = O.mass(prev, w["h"]), O.mass(cur, w["h"])
        assert abs(m1 - m0) <= 1e-12 * abs(m0)
        e0, e1 = O.energy(prev, w["h"], w["gamma"]), O.energy(cur, w["h"], w["gamma"])
        assert e1 <= e0 + 1e-14 * abs(e0)
        prev = cur
    s.close()
    if net is not None:
        net.close()
