"""The committed oracle trajectories (tests/golden/*.npz): the storage format
round-trips, and each record holds the workload, step count and solver settings
the full-size GPU parity tests assume, with the scheme's own invariants -- the
discrete energy does not increase and the mass stays at its initial value
(Sec. 3, energy stability and mass conservation of Eq. NSOP)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import goldens as G  # noqa: E402

CASES = [("hex1024_s10", "hex1024", 10), ("hex2048_s3", "hex2048", 3), ("bcc64_s50", "bcc64", 50),
         ("batch3_s100", "batch32x256", 100), ("batch22_s100", "batch32x256", 100)]


def test_whole_field_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(G, "HERE", str(tmp_path))
    rng = np.random.default_rng(0)
    phi = rng.uniform(-1.5, 1.5, size=(17, 23))
    steps = {"dt": np.array([0.01, 1.0]), "energy": np.array([2.0, 1.0])}
    G.save("t_whole", {"steps": 2, "field": "whole"}, steps, phi)
    rec = G.load("t_whole")
    assert np.abs(rec["phi"] - phi).max() <= G.QUANT_ERR
    assert G.field_error(rec, phi) <= G.QUANT_ERR
    idx = G.sample_cells((40, 64), 100, 1)
    assert idx.min() >= 0 and idx.max() < 40 * 64 and np.all(np.diff(idx) > 0)
    G.save("t_sample", {"steps": 2, "field": "sampled"}, steps, rng.uniform(size=(40, 64)), idx)
    assert G.load("t_sample")["sample_idx"].size == idx.size


@pytest.mark.parametrize("case,workload,steps", CASES)
def test_record_settings_and_invariants(case, workload, steps):
    rec = G.load(case)
    m = rec["meta"]
    assert m["workload"] == workload and m["steps"] == steps and len(rec["dt"]) == steps
    assert m["newton_rtol"] == 1e-10 and m["gmres_rtol"] == 1e-6 and m["overlap"] == 1 and m["guess"] == "phi^n"
    assert m["solver"] == ("ilu0" if workload == "bcc64" else "lu")
    assert rec["dt"][0] == m["dt_min"]  # the controller's first step (READING: dt_0 = dt_min)
    E = np.concatenate([[m["energy0"]], rec["energy"]])
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))  # energy non-increase (Sec. 3)
    assert np.abs(rec["mass"] - m["mass0"]).max() <= 1e-12 * max(1.0, abs(m["mass0"]))  # mass (Sec. 3)
    assert np.all(rec["newton_its"] >= 1) and np.all(rec["gmres_its"] >= 1)
