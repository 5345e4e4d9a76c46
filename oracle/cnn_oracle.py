"""FP64 CPU reference of the learned Newton initial guess (the periodic
convolutional network of the learned-guess form; the paper itself uses the
previous solution as the guess, Sec. 4).

TEST INFRASTRUCTURE ONLY: imported by tests and the CPU-baseline leg of
bench.py, never by the product library; shares no code with the CUDA kernels.

Network: four 3x3 periodic convolutions, channels 3 -> 32 -> 32 -> 32 -> 1, exact
GELU after the first three.  Parameters are one flat float vector laid out
layer by layer as [W (Cout, Cin, 3, 3) row-major, b (Cout)].

Features of step n -> n+1 (all from fields the solver has):
  c0 = phi^n - mean(phi^n)
  c1 = r (phi^n - phi^{n-1}),  r = dt_n / dt_{n-1}   (the extrapolation increment)
  c2 = dt_n / dt_max                                    (constant channel)
Guess: Phi_0 = phi^n + c1 + s_out * net(c), shifted by a constant so that its
mass equals that of phi^n.  Training target for net: (phi^{n+1} - phi^n - c1) / s_out.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np
from scipy.special import erf

LAYERS: List[Tuple[int, int]] = [(3, 32), (32, 32), (32, 32), (32, 1)]


def param_count() -> int:
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def unpack(theta: np.ndarray) -> List[Tuple[np.ndarray, np.ndarray]]:
    out, o = [], 0
    for ci, co in LAYERS:
        w = theta[o : o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o : o + co]
        o += co
        out.append((w, b))
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-style uniform init, deterministic."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in LAYERS:
        bound = math.sqrt(6.0 / (ci * 9))
        parts.append(rng.uniform(-bound, bound, co * ci * 9))
        parts.append(np.zeros(co))
    theta = np.concatenate(parts)
    # the last layer starts small so the initial guess is the extrapolation
    w, b = unpack(theta)[-1]
    w *= 0.01
    return theta


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[co,y,x] = b[co] + sum_{ci,dy,dx} w[co,ci,dy+1,dx+1] x[ci,(y+dy)%H,(x+dx)%W]."""
    co = w.shape[0]
    out = np.broadcast_to(b[:, None, None], (co,) + x.shape[1:]).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))  # xs[ci,y,x] = x[ci,y+dy,x+dx]
            out += np.einsum("oc,chw->ohw", w[:, :, dy + 1, dx + 1], xs)
    return out


def conv3x3_grad_input(dout: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 with respect to x."""
    ci = w.shape[1]
    dx_ = np.zeros((ci,) + dout.shape[1:])
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            t = np.einsum("oc,ohw->chw", w[:, :, dy + 1, dx + 1], dout)
            dx_ += np.roll(t, shift=(dy, dx), axis=(1, 2))
    return dx_


def conv3x3_grad_weight(x: np.ndarray, dout: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    co, ci = dout.shape[0], x.shape[0]
    dw = np.zeros((co, ci, 3, 3))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
            dw[:, :, dy + 1, dx + 1] = np.einsum("ohw,chw->oc", dout, xs)
    return dw, dout.sum(axis=(1, 2))


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta: np.ndarray, inp: np.ndarray) -> Tuple[np.ndarray, Dict]:
    """inp: (3, H, W).  Returns the network output (H, W) and the cache for backward."""
    cache = {"a": [inp], "z": []}
    a = inp
    for li, (w, b) in enumerate(unpack(theta)):
        z = conv3x3(a, w, b)
        cache["z"].append(z)
        a = gelu(z) if li < len(LAYERS) - 1 else z
        cache["a"].append(a)
    return a[0], cache


def loss_and_grad(theta: np.ndarray, inp: np.ndarray, target: np.ndarray) -> Tuple[float, np.ndarray]:
    """Mean squared error over the pixels and its gradient w.r.t. theta."""
    out, cache = forward(theta, inp)
    n = out.size
    diff = out - target
    loss = float(np.sum(diff * diff) / n)
    d = (2.0 / n) * diff[None]
    grads = []
    params = unpack(theta)
    for li in range(len(LAYERS) - 1, -1, -1):
        w, b = params[li]
        if li < len(LAYERS) - 1:
            d = d * gelu_grad(cache["z"][li])
        dw, db = conv3x3_grad_weight(cache["a"][li], d)
        grads.append((dw, db))
        d = conv3x3_grad_input(d, w)
    grads.reverse()
    flat = np.concatenate([np.concatenate([dw.ravel(), db]) for dw, db in grads])
    return loss, flat


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**t)
    vh = v / (1 - b2**t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(phin, phinm1, dt, dt_prev, dt_max) -> np.ndarray:
    r = dt / dt_prev
    return np.stack([phin - phin.mean(), r * (phin - phinm1), np.full(phin.shape, dt / dt_max)])


def target(phinp1, phin, phinm1, dt, dt_prev, s_out) -> np.ndarray:
    r = dt / dt_prev
    return (phinp1 - phin - r * (phin - phinm1)) / s_out


def guess(theta, phin, phinm1, dt, dt_prev, dt_max, s_out) -> np.ndarray:
    """Learned initial guess with the mass of phi^n."""
    c = features(phin, phinm1, dt, dt_prev, dt_max)
    out, _ = forward(theta, c)
    g = phin + c[1] + s_out * out
    return g - (g.mean() - phin.mean())
