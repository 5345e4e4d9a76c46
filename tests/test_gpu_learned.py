"""What the trained guess network gains: on a crystal-growth field it has not
seen (512^2, three hexagonal seeds, seed 3001), the learned initial guess
against the paper's phi^n start, both with BF16 subdomain factors and the same
Newton tolerance (relative to ||F(phi^n)||).  The learned run must take fewer
Newton and GMRES iterations and reach the same discrete solution: within 1e-7
in phi and 1e-9 in relative energy of the plain run, and of the FP64 oracle on
a short run."""
import math

import numpy as np
import pytest

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H, GAMMA = math.pi / 4, 0.25
PRM = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, learned, pfc as P

    build.build()
    P.lib()
    theta, s_out = learned.load()
    return P, torch, theta, s_out


def _field(shape):
    if shape[0] >= 256:
        return inputs.hex_seeds_2d(shape, H, seed=3001)
    return inputs.hex_seeds_2d(shape, H, nseeds=1, radius_cells=8, seed=3001)


def _run(P, shape, guess, theta, s_out, steps, prec=2, parts=None, stream=None):
    ny, nx = shape
    parts = parts or (nx // 16, ny // 16)
    params = P.default_params(sub=parts, overlap=1, factor_prec=prec, guess=guess, **PRM)
    s = P.Solver(shape, H, GAMMA, params, stream=stream)
    net = None
    if guess == P.PFC_GUESS_LEARNED:
        net = P.GuessNet(shape)
        net.set_params(theta)
        P.set_guess_net(s, net, s_out)
    s.set_field(_field(shape))
    infos = s.run(steps)
    phi = s.get_field()
    s.close()
    if net is not None:
        net.close()
    return phi, infos


def test_learned_guess_saves_newton_and_gmres_iterations(env):
    P, torch, theta, s_out = env
    shape = (512, 512)
    phi_p, inf_p = _run(P, shape, P.PFC_GUESS_PREV, theta, s_out, 8)
    phi_l, inf_l = _run(P, shape, P.PFC_GUESS_LEARNED, theta, s_out, 8)
    newton_p = sum(i["newton_its"] for i in inf_p[1:])
    newton_l = sum(i["newton_its"] for i in inf_l[1:])
    gmres_p = sum(i["gmres_its"] for i in inf_p[1:])
    gmres_l = sum(i["gmres_its"] for i in inf_l[1:])
    print(f"newton {newton_p} -> {newton_l}, gmres {gmres_p} -> {gmres_l}, "
          f"learned picks {[i['guess_used'] for i in inf_l]}")
    assert newton_l < newton_p and gmres_l < gmres_p
    assert any(i["guess_used"] == P.PFC_GUESS_LEARNED for i in inf_l)
    assert np.abs(phi_l - phi_p).max() <= 1e-7
    assert abs(inf_l[-1]["energy"] - inf_p[-1]["energy"]) <= 1e-9 * abs(inf_p[-1]["energy"])


def test_learned_run_matches_oracle(env):
    """Learned guess (BF16 factors) on 64^2 for 4 adaptive steps against the FP64 oracle."""
    P, torch, theta, s_out = env
    shape = (64, 64)
    phi_l, inf_l = _run(P, shape, P.PFC_GUESS_LEARNED, theta, s_out, 4)
    ref, recs = O.run(_field(shape), H, GAMMA,
                      O.Params(parts=(4, 4), overlap=1, **PRM), 4)
    assert np.abs(phi_l - ref).max() <= 1e-7
    assert abs(inf_l[-1]["energy"] - recs[-1].energy) <= 1e-9 * abs(recs[-1].energy)
    # the same run on a side stream (network on the default stream, GMRES cycles as graphs)
    phi_s, inf_s = _run(P, shape, P.PFC_GUESS_LEARNED, theta, s_out, 4, stream=torch.cuda.Stream())
    np.testing.assert_array_equal(phi_s, phi_l)
    assert [i["guess_used"] for i in inf_s] == [i["guess_used"] for i in inf_l]
