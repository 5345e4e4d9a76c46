"""Training and evaluation of the learned Newton initial guess.

Trajectories come from the solver itself (plain NKS, F32 factors) on
hexagonal-seed crystal-growth fields like the 1024^2 workload's, on a smaller
grid; every step after the first gives one sample (features of phi^n, phi^{n-1},
dt and the target correction toward phi^{n+1}), built on the device by
pfc_cnn_sample when the sample is used (only the trajectories' fields are kept).
Training runs pfc_cnn_train_step (the library's forward, backward and Adam
kernels), one sample per Adam step.  All arithmetic runs in libpfc; this module
only sequences calls and keeps the fields in device memory.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import inputs, pfc

H = math.pi / 4
GAMMA = 0.25
DT_MIN, DT_MAX, ETA = 1e-2, 10.0, 5000.0


def generate(n_traj: int, steps: int, shape=(512, 512), seed0: int = 2000, s_out: Optional[float] = None,
             sub: Optional[Tuple[int, int]] = None) -> Dict:
    """Runs n_traj trajectories of `steps` adaptive steps from seeded hexagonal
    crystal fields and returns their device fields (one sample per step after the
    first) and the output scale."""
    import torch

    ny, nx = shape
    sub = sub or (nx // 16, ny // 16)
    params = pfc.default_params(sub=sub, overlap=1, factor_prec=pfc.PFC_F32, dt_min=DT_MIN, dt_max=DT_MAX, eta=ETA)
    solver = pfc.Solver(shape, H, GAMMA, params)
    net = pfc.GuessNet(shape)
    raw: List[Tuple] = []
    t0 = time.perf_counter()
    for tr in range(n_traj):
        phi0 = inputs.hex_seeds_2d(shape, H, seed=seed0 + tr)
        solver.set_field(phi0)
        hist = [solver.get_field_device()]
        dts = []
        for _ in range(steps):
            dt = solver.next_dt()
            for cut in range(4):  # a failed step leaves phi^n as it was: retry with dt / 2
                try:
                    solver.step(dt)
                    break
                except pfc.PfcError:
                    if cut == 3:
                        raise
                    dt *= 0.5
            dts.append(dt)
            hist.append(solver.get_field_device())
        for k in range(1, steps):  # sample: phi^{k-1}, phi^k -> phi^{k+1}, dt_k, dt_{k-1}
            raw.append((hist[k - 1], hist[k], hist[k + 1], dts[k] / dts[k - 1], dts[k] / DT_MAX))
    if s_out is None:  # output scale: rms of the extrapolation error over the first trajectory's samples
        errs = []
        for a, b, c, r, _ in raw[: max(1, steps - 1)]:
            e = (c - b - r * (b - a)).cpu().numpy()
            errs.append(float(np.sqrt(np.mean(e * e))))
        s_out = float(np.mean(errs)) or 1e-3
    solver.close()
    return {"raw": raw, "s_out": s_out, "shape": tuple(shape), "gen_seconds": time.perf_counter() - t0, "net": net}


class _Samples:
    """Sample i of a generate() result, built on the device into two reused buffers."""

    def __init__(self, data: Dict):
        import torch

        self.data = data
        self.f = torch.empty((3,) + tuple(data["shape"]), dtype=torch.float64, device="cuda")
        self.t = torch.empty(tuple(data["shape"]), dtype=torch.float64, device="cuda")

    def __len__(self) -> int:
        return len(self.data["raw"])

    def __getitem__(self, i: int):
        a, b, c, r, c2 = self.data["raw"][i]
        self.data["net"].sample(a, b, c, r, c2, self.data["s_out"], self.f, self.t)
        return self.f, self.t


def _init_params(seed: int) -> np.ndarray:
    """He-style uniform initialisation; the last layer starts near zero so the
    first guesses are the extrapolation."""
    rng = np.random.default_rng(seed)
    parts = []
    layers = [(3, 32), (32, 32), (32, 32), (32, 1)]
    for li, (ci, co) in enumerate(layers):
        bound = math.sqrt(6.0 / (ci * 9))
        w = rng.uniform(-bound, bound, co * ci * 9)
        if li == len(layers) - 1:
            w *= 0.01
        parts.append(w)
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def train_net(data: Dict, epochs: int = 3, lr: float = 1e-3, seed: int = 0,
              theta0: Optional[np.ndarray] = None, lr_min: Optional[float] = None,
              holdout: int = 0) -> Tuple[np.ndarray, List[float]]:
    """Adam on single samples in a seeded random order, the step size following
    a cosine from lr to lr_min (constant when lr_min is None).  The last
    `holdout` samples are not trained on; the history holds per epoch the mean
    training loss and, with a hold-out, the mean hold-out loss."""
    net: pfc.GuessNet = data["net"]
    net.set_params(theta0 if theta0 is not None else _init_params(seed))
    rng = np.random.default_rng(seed)
    samples = _Samples(data)
    n = len(samples) - holdout
    total = epochs * n
    t = 0
    history = []
    for _ in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for i in order:
            t += 1
            a = lr if lr_min is None else lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * (t - 1) / total))
            tot += net.train_step(*samples[i], a, t)
        rec = {"train": tot / max(n, 1)}
        if holdout:
            rec["holdout"] = sum(net.loss_grad(*samples[i])[0] for i in range(n, n + holdout)) / holdout
        history.append(rec)
    return net.get_params(), history


# The committed network: trajectories of the 1024^2 workload's distribution (three hexagonal
# seeds, gamma 0.25, adaptive dt) on 512^2 grids, their first 25 steps (the growth stage the
# 1024^2 workload's timed steps are in).
DEFAULT_RECIPE = dict(n_traj=96, steps=25, size=512, epochs=20, lr=3e-4, lr_min=3e-5, seed=0, seed0=2000)
WEIGHTS = "guess_net.npz"


def train_default(out_path: str, **over) -> Dict:
    """Generates the trajectories, trains, and saves theta, s_out and the recipe to out_path (.npz)."""
    import torch

    rc = dict(DEFAULT_RECIPE, **over)
    t0 = time.perf_counter()
    data = generate(rc["n_traj"], rc["steps"], shape=(rc["size"], rc["size"]), seed0=rc["seed0"])
    hold = rc["steps"] - 1  # the last trajectory's samples
    theta, hist = train_net(data, epochs=rc["epochs"], lr=rc["lr"], lr_min=rc["lr_min"], seed=rc["seed"],
                            holdout=hold)
    info = {"recipe": rc, "s_out": data["s_out"], "history": hist, "samples": len(data["raw"]) - hold,
            "gen_seconds": data["gen_seconds"], "seconds": time.perf_counter() - t0}
    np.savez(out_path, theta=theta.astype(np.float32), s_out=np.array([data["s_out"]]),
             info=np.array(json.dumps(info)))
    data["net"].close()
    del data
    torch.cuda.empty_cache()
    return info


def load(path: Optional[str] = None) -> Tuple[np.ndarray, float]:
    """theta and s_out of a saved network (default: the committed one)."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", WEIGHTS)
    z = np.load(path)
    return z["theta"].astype(np.float32), float(z["s_out"][0])


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description="train the learned Newton initial guess on solver trajectories")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", WEIGHTS))
    for k, v in DEFAULT_RECIPE.items():
        ap.add_argument("--" + k.replace("_", "-"), type=type(v), default=v)
    args = ap.parse_args()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    over = {k: getattr(args, k) for k in DEFAULT_RECIPE}
    print(json.dumps(train_default(args.out, **over)))


def evaluate(theta: np.ndarray, s_out: float, shape=(1024, 1024), steps: int = 12, warmup: int = 3,
             seed: int = 1001, factor_prec: int = pfc.PFC_BF16, modes=("prev", "extrap", "learned")) -> Dict:
    """Newton / GMRES iterations and time per step with phi^n, the extrapolated
    guess and the learned guess (safeguards included) on a hexagonal-seed field."""
    import torch

    ny, nx = shape
    out = {}
    phi0 = inputs.hex_seeds_2d(shape, H, seed=seed)
    for mode in modes:
        guess = {"prev": pfc.PFC_GUESS_PREV, "extrap": pfc.PFC_GUESS_EXTRAP, "learned": pfc.PFC_GUESS_LEARNED}[mode]
        params = pfc.default_params(sub=(nx // 16, ny // 16), overlap=1, factor_prec=factor_prec, guess=guess,
                                    dt_min=DT_MIN, dt_max=DT_MAX, eta=ETA)
        s = pfc.Solver(shape, H, GAMMA, params)
        net = None
        if mode == "learned":
            net = pfc.GuessNet(shape)
            net.set_params(theta)
            pfc.set_guess_net(s, net, s_out)
        s.set_field(phi0)
        s.run(warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = s.run(steps)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out[mode] = {"steps_per_s": steps / el, "newton_per_step": sum(i["newton_its"] for i in infos) / steps,
                     "gmres_per_step": sum(i["gmres_its"] for i in infos) / steps,
                     "guess_used": [i["guess_used"] for i in infos],
                     "newton_its": [i["newton_its"] for i in infos], "dt": [i["dt"] for i in infos],
                     "energy_last": infos[-1]["energy"], "field": s.get_field()}
        s.close()
        if net is not None:
            net.close()
    return out
