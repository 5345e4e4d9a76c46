"""Writes the oracle trajectories the full-size GPU parity tests compare against.

Calls only the FP64 CPU oracle (oracle/pfc_oracle.py) on the seeded initial
fields of paper_1703_01202_gb300/inputs.py; nothing here runs or reads the CUDA
path.  Each case is one run of the workload's adaptive time stepping (Eq.
sencondt) with the paper's method: inexact Newton (Sec. 4, Eq. newton),
right-preconditioned GMRES(30) (Eq. hjacobi) and left-RAS (Eq. ras) with exact
block LU in 2D and shifted ILU(0) in 3D, Newton rtol 1e-10, GMRES rtol 1e-6,
starting every Newton solve from phi^n (Sec. 4).

    python tests/golden/make_goldens.py [case ...]     # default: every case

Cases (grid, steps; what the record keeps):
  hex1024_s10     1024^2 crystal growth, 64 x 64 cores, first 10 adaptive steps; whole field
  hex2048_s3      2048^2, 128 x 128 cores, first 3 adaptive steps; sampled cells: 4 rows, 4 columns,
                  49,152 random cells and every cell the steps moved by more than 1e-13
  bcc64_s50       64^3 BCC growth, 7 x 7 x 7 uneven cores, ILU(0), 50 adaptive steps; whole field
  batch3_s100     ensemble member 3 (256^2 noise, gamma_3), 16 x 16 cores, 100 steps; whole field
  batch22_s100    ensemble member 22, likewise
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import goldens  # noqa: E402
from oracle import pfc_oracle as O  # noqa: E402
from paper_1703_01202_gb300 import inputs  # noqa: E402


def case_setup(case: str):
    """(initial field, h, gamma, oracle Params, steps, workload name, whole field?)"""
    if case.startswith("batch"):
        member = int(case[len("batch"):].split("_")[0])
        w = inputs.workload("batch32x256")
        p = O.Params(parts=w["parts"], overlap=1, dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"])
        return w["phis"][member], w["h"], w["gammas"][member], p, 100, "batch32x256", True, {"member": member}
    name, steps = case.split("_s")
    w = inputs.workload(name)
    p = O.Params(parts=w["parts"], overlap=1, dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"])
    if len(w["shape"]) == 3:
        p.subdomain_solver = "ilu0"
        p.ilu_shift = 0.1
    return w["phi"], w["h"], w["gamma"], p, int(steps), name, name != "hex2048", {}


def make(case: str) -> None:
    phi0, h, gamma, p, steps, wname, whole, extra = case_setup(case)
    t0 = time.time()
    phi, recs = O.run(phi0, h, gamma, p, steps)
    secs = time.time() - t0
    per_step = {
        "dt": np.array([r.dt for r in recs]),
        "energy": np.array([r.energy for r in recs]),
        "mass": np.array([r.mass for r in recs]),
        "newton_its": np.array([r.newton_its for r in recs], dtype=np.int32),
        "gmres_its": np.array([r.gmres_its for r in recs], dtype=np.int32),
    }
    meta = dict(case=case, workload=wname, steps=steps, h=h, gamma=gamma, parts=list(p.parts), overlap=p.overlap,
                solver=p.subdomain_solver, ilu_shift=p.ilu_shift, newton_rtol=p.newton_rtol,
                gmres_rtol=p.gmres_rtol, dt_min=p.dt_min, dt_max=p.dt_max, eta=p.eta, guess="phi^n",
                mass0=O.mass(phi0, h), energy0=O.energy(phi0, h, gamma), oracle_seconds=round(secs, 1),
                field="whole" if whole else "sampled", **extra)
    sample = None
    if not whole:  # the spread sample plus every cell the steps moved (the growing crystals), largest first
        moved = np.flatnonzero(np.abs(phi - phi0).ravel() > 1e-13)
        if moved.size > 400000:
            moved = moved[np.argsort(-np.abs(phi - phi0).ravel()[moved], kind="stable")[:400000]]
        sample = np.union1d(goldens.sample_cells(phi.shape, 49152, 4242), moved).astype(np.int64)
        meta["moved_cells"] = int(moved.size)
    goldens.save(case, meta, per_step, phi, sample)
    print(f"{case}: {steps} steps in {secs:.0f} s, dt[-1] = {recs[-1].dt:.6g}, "
          f"newton {per_step['newton_its'].tolist()}, gmres {per_step['gmres_its'].tolist()}", flush=True)


CASES = ["hex1024_s10", "hex2048_s3", "bcc64_s50", "batch3_s100", "batch22_s100"]

if __name__ == "__main__":
    for c in sys.argv[1:] or CASES:
        make(c)
