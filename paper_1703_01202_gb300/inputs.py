"""Seeded synthetic inputs: initial fields for the PFC time stepper.

This module holds no arithmetic of the method (no stencil, energy or solver);
it only builds initial density fields from the crystal profiles the paper
uses to set up its tests, and a portable counter-based random generator.
Both the CUDA path (through the C-ABI) and the CPU oracle are fed the arrays
it returns; neither side generates its own inputs.

Arrays are float64 with shape (Ny, Nx) or (Nz, Ny, Nx): x is the last
(fastest) axis.  Cell centres sit at ((i + 1/2) h, (j + 1/2) h[, (k + 1/2) h])
for 0-based indices (Sec. 3, cell-centred grid).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` outputs of the SplitMix64 generator (Steele, Lea & Flood 2014)
    started from `seed`: state += 0x9E3779B97F4A7C15, then the published
    xor-shift-multiply finaliser.  Returns uint64."""
    golden = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + golden * (np.arange(1, count + 1, dtype=np.uint64))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def cell_centres(shape: Sequence[int], h: float) -> List[np.ndarray]:
    """Broadcastable coordinate arrays in array-axis order (last axis = x)."""
    out = []
    nd = len(shape)
    for ax, n in enumerate(shape):
        c = (np.arange(n, dtype=np.float64) + 0.5) * h
        sh = [1] * nd
        sh[ax] = n
        out.append(c.reshape(sh))
    return out


def noise_field(shape: Sequence[int], mean: float, amp: float, seed: int) -> np.ndarray:
    """phi = mean + amp * U(-1, 1) i.i.d. per point (test A's random liquid)."""
    n = int(np.prod(shape))
    return (mean + amp * uniform(seed, n, -1.0, 1.0)).reshape(tuple(shape))


def sine_field(shape: Sequence[int], h: float, amp: float = 0.5, period: float = 32.0) -> np.ndarray:
    """Smooth product of sines used for the grid-convergence study (Sec. 5, test A)."""
    coords = cell_centres(shape, h)
    out = np.full(tuple(shape), amp)
    for c in coords:
        out = out * np.sin(2.0 * math.pi * c / period)
    return out


def _periodic_dist(a: np.ndarray, b: np.ndarray, L: np.ndarray) -> float:
    d = np.abs(a - b)
    d = np.minimum(d, L - d)
    return float(np.sqrt(np.sum(d * d)))


def _place_centres(count: int, L: np.ndarray, min_dist: float, seed: int) -> List[np.ndarray]:
    """Uniform random centres, rejecting any closer than `min_dist` (periodic)."""
    centres: List[np.ndarray] = []
    draw = 0
    while len(centres) < count:
        u = uniform(seed * 7919 + 17, 64 * len(L), 0.0, 1.0)
        for t in range(64):
            c = u[t * len(L) : (t + 1) * len(L)] * L
            draw += 1
            if all(_periodic_dist(c, o, L) >= min_dist for o in centres):
                centres.append(c)
                if len(centres) == count:
                    break
        seed += 1
        if draw > 100000:
            raise RuntimeError("could not place seeds without overlap")
    return centres


def hex_seeds_2d(
    shape: Tuple[int, int],
    h: float,
    mean: float = 0.285,
    nseeds: int = 3,
    radius_cells: float = 20.0,
    q: float = math.sqrt(3.0) / 2.0,
    amp: float = 0.446,
    seed: int = 1001,
) -> np.ndarray:
    """Background density `mean` with `nseeds` randomly placed, randomly rotated
    discs carrying the one-mode hexagonal profile
        mean + A (cos(q xr) cos(q yr / sqrt3) - cos(2 q yr / sqrt3) / 2)
    (test B's crystallite profile), xr, yr being coordinates rotated by omega
    about the disc centre.  Discs do not overlap (periodic distance >= 2 r)."""
    ny, nx = shape
    L = np.array([ny * h, nx * h])
    r = radius_cells * h
    centres = _place_centres(nseeds, L, 2.0 * r, seed)
    angles = uniform(seed * 31 + 5, nseeds, 0.0, math.pi / 3.0)
    y, x = cell_centres(shape, h)
    phi = np.full(shape, mean, dtype=np.float64)
    for c, om in zip(centres, angles):
        dy = y - c[0]
        dx = x - c[1]
        dy = dy - L[0] * np.round(dy / L[0])
        dx = dx - L[1] * np.round(dx / L[1])
        xr = math.cos(om) * dx - math.sin(om) * dy
        yr = math.sin(om) * dx + math.cos(om) * dy
        inside = dx * dx + dy * dy <= r * r
        prof = mean + amp * (np.cos(q * xr) * np.cos(q * yr / math.sqrt(3.0)) - 0.5 * np.cos(2.0 * q * yr / math.sqrt(3.0)))
        phi = np.where(inside, prof, phi)
    return phi


def bcc_seeds_3d(
    shape: Tuple[int, int, int],
    h: float,
    mean: float = -0.325,
    nseeds: int = 4,
    d0: float = 5.0 * math.pi,
    q: float = 1.0 / math.sqrt(2.0),
    amp: float = 1.0,
    seed: int = 1003,
) -> np.ndarray:
    """Background `mean` plus `nseeds` spheres of radius d0 carrying the BCC mode
    cos(xq)cos(yq) + cos(xq)cos(zq) + cos(yq)cos(zq), tapered by
    rho = (1 - (r/d0)^2)^2 inside the sphere, in local coordinates rotated by a
    random omega about z (test D's crystallites; random centres, no overlap)."""
    nz, ny, nx = shape
    L = np.array([nz * h, ny * h, nx * h])
    centres = _place_centres(nseeds, L, 2.0 * d0, seed)
    angles = uniform(seed * 31 + 5, nseeds, 0.0, 2.0 * math.pi)
    z, y, x = cell_centres(shape, h)
    phi = np.full(shape, mean, dtype=np.float64)
    for c, om in zip(centres, angles):
        dz = z - c[0]
        dy = y - c[1]
        dx = x - c[2]
        dz = dz - L[0] * np.round(dz / L[0])
        dy = dy - L[1] * np.round(dy / L[1])
        dx = dx - L[2] * np.round(dx / L[2])
        xr = math.cos(om) * dx - math.sin(om) * dy
        yr = math.sin(om) * dx + math.cos(om) * dy
        zr = dz
        rr2 = (dx * dx + dy * dy + dz * dz) / (d0 * d0)
        rho = np.where(rr2 <= 1.0, (1.0 - rr2) ** 2, 0.0)
        bcc = np.cos(xr * q) * np.cos(yr * q) + np.cos(xr * q) * np.cos(zr * q) + np.cos(yr * q) * np.cos(zr * q)
        phi = phi + amp * rho * bcc
    return phi


def crack_field(
    shape: Tuple[int, int],
    h: float,
    mean: float = 0.49,
    qx: float = math.sqrt(3.0) / 2.0,
    stretch: float = 0.9,
    notch_cells: Tuple[int, int] = (20, 40),
    notch_value: float = 0.79,
) -> np.ndarray:
    """Test C's initial state: a stretched one-mode hexagonal lattice
        mean + cos(qy y / sqrt3) cos(qx x) - cos(2 qy y / sqrt3) / 2,  qy = stretch * qx,
    on every cell, with a centred notch of notch_cells (rows, columns) replaced by the
    coexisting liquid density notch_value."""
    ny, nx = shape
    qy = stretch * qx
    y, x = cell_centres(shape, h)
    phi = mean + np.cos(qy * y / math.sqrt(3.0)) * np.cos(qx * x) - 0.5 * np.cos(2.0 * qy * y / math.sqrt(3.0))
    phi = np.broadcast_to(phi, shape).copy()
    ry, rx = notch_cells
    y0, x0 = (ny - ry) // 2, (nx - rx) // 2
    phi[y0 : y0 + ry, x0 : x0 + rx] = notch_value
    return phi


# Named workloads (shape in array-axis order, h, gamma, generator).  The sizes
# and physical parameters are those of the crystal-growth workloads; the
# solver settings live with the callers.
def workload(name: str) -> dict:
    if name == "noise64":  # 64^2 liquid from noise, fixed dt 0.1 x 20 steps
        return dict(shape=(64, 64), h=math.pi / 4, gamma=0.25, phi=noise_field((64, 64), 0.07, 0.07, 1000),
                    parts=(4, 4), fixed_dt=0.1, steps=20)
    if name == "hex1024":  # 1024^2 crystal growth from 3 hexagonal seeds, adaptive dt
        return dict(shape=(1024, 1024), h=math.pi / 4, gamma=0.25, phi=hex_seeds_2d((1024, 1024), math.pi / 4, seed=1001),
                    parts=(64, 64), dt_min=1e-2, dt_max=10.0, eta=5000.0, steps=500)
    if name == "hex2048":
        return dict(shape=(2048, 2048), h=math.pi / 4, gamma=0.25,
                    phi=hex_seeds_2d((2048, 2048), math.pi / 4, seed=1002),
                    parts=(128, 128), dt_min=1e-2, dt_max=10.0, eta=5000.0, steps=20)
    if name == "bcc256":
        h = 80.0 * math.pi / 256.0
        return dict(shape=(256, 256, 256), h=h, gamma=0.3, phi=bcc_seeds_3d((256, 256, 256), h, seed=1003),
                    parts=(7, 7, 7), dt_min=0.5, dt_max=10.0, eta=500.0, steps=50)
    if name == "bcc64":  # the 3D recipe on a 64^3 grid (same h, gamma, mean, taper; seed radius halved)
        h = 80.0 * math.pi / 256.0
        return dict(shape=(64, 64, 64), h=h, gamma=0.3,
                    phi=bcc_seeds_3d((64, 64, 64), h, nseeds=4, d0=2.5 * math.pi, seed=1005),
                    parts=(7, 7, 7), dt_min=0.5, dt_max=10.0, eta=500.0, steps=50)
    if name == "batch32x256":  # 32 independent 256^2 noise runs, gamma_i ~ U(0.1, 0.35), adaptive dt
        gammas = uniform(1004 * 7 + 3, 32, 0.1, 0.35)
        return dict(shape=(256, 256), h=math.pi / 4, gammas=[float(g) for g in gammas],
                    phis=[noise_field((256, 256), 0.07, 0.07, 1004 + i) for i in range(32)],
                    parts=(16, 16), dt_min=1e-2, dt_max=10.0, eta=5000.0, steps=100)
    if name == "crack4096x1024":  # crack propagation in a stretched crystal, gamma = 1, adaptive dt in [1, 5]
        h = math.pi / 3.0
        return dict(shape=(1024, 4096), h=h, gamma=1.0, phi=crack_field((1024, 4096), h),
                    parts=(64, 256), dt_min=1.0, dt_max=5.0, eta=100.0, steps=3200)
    if name == "crack128x48":  # the same recipe on a 128 x 48 grid (the notch keeps its 40 x 20 cells)
        h = math.pi / 3.0
        return dict(shape=(48, 128), h=h, gamma=1.0, phi=crack_field((48, 128), h),
                    parts=(3, 8), dt_min=1.0, dt_max=5.0, eta=100.0, steps=20)
    raise KeyError(name)
