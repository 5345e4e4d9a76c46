"""GPU parity of the learned-guess network kernels (BF16 weights and
activations, FP32 accumulation) against the FP64 reference -- per output pixel,
per gradient entry, and against finite differences -- and the learned guess
inside the time step."""
import math

import numpy as np
import pytest

from oracle import cnn_oracle as C
from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P, torch


def sample(shape, seed):
    rng = np.random.default_rng(seed)
    feat = np.stack([rng.normal(scale=0.3, size=shape), rng.normal(scale=0.05, size=shape), np.full(shape, 0.7)])
    tgt = rng.normal(size=shape)
    theta = C.init_params(seed)
    theta[-(32 * 9 + 1):] = rng.normal(scale=0.1, size=32 * 9 + 1)
    return feat, tgt, theta


def bf16_weights(theta):
    """The parameters as the network holds them for its arithmetic: weights rounded to BF16
    (round to nearest even), biases in FP32; returned in FP64 for the reference."""
    out = theta.astype(np.float32).copy()
    for li, (ci, co) in enumerate(C.LAYERS):
        lo = sum(c2 * c1 * 9 + c2 for c1, c2 in C.LAYERS[:li])
        w = out[lo : lo + co * ci * 9].view(np.uint32)
        w[:] = (w + np.uint32(0x7FFF) + ((w >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return out.astype(np.float64)


def layer_slices():
    for li, (ci, co) in enumerate(C.LAYERS):
        lo = sum(c2 * c1 * 9 + c2 for c1, c2 in C.LAYERS[:li])
        yield li, slice(lo, lo + co * ci * 9 + co)


@pytest.mark.parametrize("shape", [(24, 20), (33, 17)])
def test_forward_matches_fp64_reference(env, shape):
    """Every pixel of the BF16 network's output against the FP64 reference evaluated with the
    same (BF16-rounded) weights: the remaining difference is the BF16 rounding of the
    activations (2^-9 relative per layer), bounded here at 1e-2 of the largest output."""
    P, torch = env
    feat, _, theta = sample(shape, 1)
    net = P.GuessNet(shape)
    net.set_params(theta)
    out = net.forward(torch.from_numpy(feat).cuda()).cpu().numpy()
    ref, _ = C.forward(bf16_weights(theta), feat)
    assert np.abs(out - ref).max() <= 1e-2 * np.abs(ref).max()
    ref32, _ = C.forward(theta.astype(np.float32).astype(np.float64), feat)  # unrounded weights too
    assert np.abs(out - ref32).max() <= 2e-2 * np.abs(ref32).max()


def test_gradient_matches_fp64_reference(env):
    """Every entry of the loss gradient (backward kernels) against the FP64 reference with the
    same weights, within 1e-2 of the largest entry of its layer."""
    P, torch = env
    shape = (32, 24)
    feat, tgt, theta = sample(shape, 2)
    net = P.GuessNet(shape)
    net.set_params(theta)
    loss, g = net.loss_grad(torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda())
    rl, rg = C.loss_and_grad(bf16_weights(theta), feat, tgt)
    assert loss == pytest.approx(rl, rel=1e-2)
    for li, sl in layer_slices():
        assert np.abs(g[sl] - rg[sl]).max() <= 1e-2 * np.abs(rg[sl]).max(), li


def test_gradient_entries_match_finite_differences(env):
    """Eight GPU gradient entries (two per layer, seeded) against central differences of the
    FP64 reference loss, (L(theta + e) - L(theta - e)) / 2e with e = 1e-4 (its truncation error
    is O(e^2), far below the bound), within 1e-2 of the largest gradient entry of the layer."""
    P, torch = env
    shape = (32, 24)
    feat, tgt, theta = sample(shape, 4)
    net = P.GuessNet(shape)
    net.set_params(theta)
    _, g = net.loss_grad(torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda())
    base = bf16_weights(theta)
    rng = np.random.default_rng(5)
    for li, sl in layer_slices():
        gmax = np.abs(g[sl]).max()
        for k in rng.choice(np.arange(sl.start, sl.stop), size=2, replace=False):
            eps = 1e-4
            tp, tm = base.copy(), base.copy()
            tp[k] += eps
            tm[k] -= eps
            fd = (C.loss_and_grad(tp, feat, tgt)[0] - C.loss_and_grad(tm, feat, tgt)[0]) / (2 * eps)
            assert abs(g[k] - fd) <= 1e-2 * gmax, (li, int(k), float(g[k]), fd)


def test_adam_training_reduces_the_loss(env):
    P, torch = env
    shape = (32, 32)
    feat, _, theta = sample(shape, 3)
    # a target the network can represent: a smooth function of the inputs
    tgt = np.tanh(3.0 * feat[0]) + 0.5 * feat[1] / 0.05
    net = P.GuessNet(shape)
    net.set_params(theta)
    f, t = torch.from_numpy(feat).cuda(), torch.from_numpy(tgt).cuda()
    losses = [net.train_step(f, t, 3e-3, i + 1) for i in range(60)]
    assert losses[-1] < 0.5 * losses[0]


def test_learned_guess_with_zero_network_is_the_extrapolation(env):
    """All-zero parameters make the network output zero, so the learned guess
    equals the extrapolated one and the step matches the extrapolation run."""
    P, torch = env
    shape = (48, 48)
    h, gamma = math.pi / 4, 0.25
    phi0 = inputs.hex_seeds_2d(shape, h, nseeds=1, radius_cells=8, seed=4)
    prm = dict(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0)
    a = P.Solver(shape, h, gamma, P.default_params(guess=P.PFC_GUESS_LEARNED, **prm))
    b = P.Solver(shape, h, gamma, P.default_params(guess=P.PFC_GUESS_EXTRAP, **prm))
    net = P.GuessNet(shape)
    net.set_params(np.zeros(P.GuessNet.param_count(), dtype=np.float32))
    P.set_guess_net(a, net, 0.01)
    a.set_field(phi0)
    b.set_field(phi0)
    ia, ib = a.run(4), b.run(4)
    # step 0 has no history (phi^n); afterwards the learned and extrapolated guesses tie,
    # the tie keeps the extrapolation, and the safeguard picks as in the extrapolation run
    ga, gb = [i["guess_used"] for i in ia], [i["guess_used"] for i in ib]
    assert ga[0] == P.PFC_GUESS_PREV and ga == gb and P.PFC_GUESS_LEARNED not in ga
    np.testing.assert_allclose(a.get_field(), b.get_field(), rtol=0, atol=1e-10)
    # the oracle's run with the extrapolated guess agrees too
    ref, _ = O.run(phi0, h, gamma, O.Params(parts=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0), 4,
                   guess="extrap")
    assert np.abs(a.get_field() - ref).max() <= 1e-8
