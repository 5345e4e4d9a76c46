"""Storage format of the oracle trajectories in tests/golden/*.npz.

This module only encodes and decodes arrays; it holds none of the method's
arithmetic and never calls the oracle.  The files are written by
make_goldens.py (which calls oracle/ only) and read by the GPU parity tests
and by bench.py's error report.

A record holds the oracle's per-step scalars of one workload run (dt, energy,
mass, Newton and GMRES iterations) and its final field phi, either
  * whole: phi rounded to the nearest multiple of 2^-32 (2.3e-10, far below the
    1e-8 parity tolerance) and stored as int64 with its bytes regrouped by
    significance so that zlib finds the long runs, or
  * sampled: phi at a set of cells (exact float64 values), for grids too
    large to store whole -- rows, columns and random cells spread over the
    grid plus every cell the run moved; and sum, sum of squares, min and max
    of the whole field.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
QUANT = 2.0 ** 32  # whole fields: phi * QUANT rounded to an integer
QUANT_ERR = 0.5 / QUANT  # largest rounding error of a stored whole field


def path_of(name: str) -> str:
    return os.path.join(HERE, name + ".npz")


def _pack_whole(phi: np.ndarray) -> np.ndarray:
    q = np.rint(phi.ravel() * QUANT).astype("<i8")
    return np.ascontiguousarray(q.view(np.uint8).reshape(-1, 8).T)


def _unpack_whole(b: np.ndarray, shape) -> np.ndarray:
    q = np.ascontiguousarray(b.T).reshape(-1).view("<i8")
    return (q.astype(np.float64) / QUANT).reshape(shape)


def sample_cells(shape, count: int, seed: int) -> np.ndarray:
    """Flat indices of the sampled cells: every cell of 4 rows and 4 columns spread
    over the grid plus `count` cells drawn by SplitMix64 (x fastest, sorted, unique)."""
    from paper_1703_01202_gb300 import inputs

    ny, nx = shape[-2], shape[-1]
    n = int(np.prod(shape))
    rows = [(k * ny) // 4 + 1 for k in range(4)]
    cols = [(k * nx) // 4 + 2 for k in range(4)]
    idx = [r * nx + np.arange(nx) for r in rows] + [np.arange(ny) * nx + c for c in cols]
    draw = (inputs.uniform(seed, count) * n).astype(np.int64)
    return np.unique(np.concatenate(idx + [np.minimum(draw, n - 1)])).astype(np.int64)


def save(name: str, meta: Dict, steps: Dict[str, np.ndarray], phi: np.ndarray, sample: Optional[np.ndarray] = None):
    arrays = {k: np.asarray(v) for k, v in steps.items()}
    arrays["meta"] = np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)
    arrays["shape"] = np.asarray(phi.shape, dtype=np.int64)
    arrays["stats"] = np.array([phi.sum(), np.square(phi).sum(), phi.min(), phi.max()])
    if sample is None:
        arrays["whole"] = _pack_whole(phi)
    else:
        arrays["sample_idx"] = sample
        arrays["sample_val"] = phi.ravel()[sample]
    np.savez_compressed(path_of(name), **arrays)


def load(name: str) -> Dict:
    """{'meta', 'shape', 'stats', per-step arrays, and 'phi' (whole field) or
    'sample_idx' / 'sample_val'}."""
    with np.load(path_of(name)) as z:
        out = {k: z[k] for k in z.files if k not in ("meta", "whole")}
        out["meta"] = json.loads(bytes(z["meta"]).decode())
        out["shape"] = tuple(int(v) for v in z["shape"])
        if "whole" in z.files:
            out["phi"] = _unpack_whole(z["whole"], out["shape"])
    return out


def field_error(rec: Dict, phi: np.ndarray) -> float:
    """max |phi - phi_oracle| over the stored cells (all cells of a whole record)."""
    if "phi" in rec:
        return float(np.abs(phi - rec["phi"]).max())
    return float(np.abs(phi.ravel()[rec["sample_idx"]] - rec["sample_val"]).max())
