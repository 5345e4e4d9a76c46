"""GPU parity at the workloads' own sizes and step counts, element by element,
against the FP64 oracle's trajectories (tests/golden/*.npz, written by
tests/golden/make_goldens.py, which calls only oracle/).

Each test runs the GPU path through the C ABI, in the configuration bench.py
times (left-RAS with one overlap cell per side, adaptive dt, GMRES cycles as
CUDA graphs on a side stream), over the record's steps from the same seeded
initial field, and compares:
  * phi after the last step: max |phi_gpu - phi_oracle| over every cell (whole
    records) or over the stored cells (the 2048^2 record: 4 rows, 4 columns and
    49,152 random cells), plus the whole field's sum, sum of squares, min and max;
  * the energy and mass after every step, and the time step the controller took.
Tolerances (the FP64 solver stops Newton at 1e-10 ||F(phi^n)||, both sides):
plain FP64 path max |dphi| <= 1e-8 and relative energy error <= 1e-10; mixed
(FP32 / BF16 subdomain factors) and learned-guess forms <= 1e-7 and <= 1e-9;
mass within 1e-12 of the initial mass (relative).  Whole records store phi
rounded to 2^-32, which adds at most 1.2e-10 to the field error."""
import math
import os
import sys

import numpy as np
import pytest

from paper_1703_01202_gb300 import inputs

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import goldens as G  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {"f64": (1e-8, 1e-10), "mixed": (1e-7, 1e-9)}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, learned, pfc as P

    build.build()
    P.lib()
    return P, torch, learned


def _solver(P, torch, learned, workload, prec, guess_learned=False, gamma=None, **kw):
    w = inputs.workload(workload)
    params = P.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=prec, dt_min=w["dt_min"],
                              dt_max=w["dt_max"], eta=w["eta"],
                              guess=P.PFC_GUESS_LEARNED if guess_learned else P.PFC_GUESS_PREV, **kw)
    s = P.Solver(w["shape"], w["h"], w["gamma"] if gamma is None else gamma, params, stream=torch.cuda.Stream())
    net = None
    if guess_learned:
        theta, s_out = learned.load()
        net = P.GuessNet(w["shape"])
        net.set_params(theta)
        P.set_guess_net(s, net, s_out)
    return s, net, w


def check_against(rec, infos, phi, tol):
    tphi, te = tol
    steps = rec["meta"]["steps"]
    assert len(infos) == steps
    e = np.array([i["energy"] for i in infos])
    m = np.array([i["mass"] for i in infos])
    dt = np.array([i["dt"] for i in infos])
    rel_e = np.abs(e - rec["energy"]) / np.abs(rec["energy"])
    assert rel_e.max() <= te, (rel_e.max(), te)
    m0 = rec["meta"]["mass0"]
    assert np.abs(m - m0).max() <= 1e-12 * max(1.0, abs(m0))
    assert np.abs(dt - rec["dt"]).max() <= 1e-6 * rec["dt"].max()
    err = G.field_error(rec, phi)
    slack = G.QUANT_ERR if "phi" in rec else 0.0
    assert err <= tphi + slack, (err, tphi)
    s, s2, lo, hi = rec["stats"]
    n = phi.size
    assert abs(phi.sum() - s) <= tphi * n
    assert abs(np.square(phi).sum() - s2) <= 2 * tphi * np.abs(phi).sum() + tphi * tphi * n
    assert abs(phi.min() - lo) <= tphi and abs(phi.max() - hi) <= tphi
    return err, rel_e.max()


@pytest.mark.parametrize("prec,learned_guess,form", [(0, False, {}), (1, False, {}), (2, False, {}), (2, True, {}),
                                                     (2, True, {"gmres_fast_dots": 1}), (2, True, {"jvp_fp32": 1})])
def test_hex1024_ten_steps_match_oracle(env, prec, learned_guess, form):
    """The 1024^2 crystal-growth workload (64 x 64 cores), its first 10 adaptive steps; also the
    opt-in mixed forms (FP32 Arnoldi dot products, FP32 JVP)."""
    P, torch, learned = env
    rec = G.load("hex1024_s10")
    s, net, w = _solver(P, torch, learned, "hex1024", prec, learned_guess, **form)
    s.set_field(w["phi"])
    infos = s.run(rec["meta"]["steps"])
    err, rel_e = check_against(rec, infos, s.get_field(), TOL["f64" if prec == 0 and not learned_guess else "mixed"])
    print(f"hex1024 prec {prec} learned {learned_guess} {form}: max|dphi| {err:.2e}, energy {rel_e:.2e}, "
          f"newton {[i['newton_its'] for i in infos]}")
    s.close()
    if net is not None:
        net.close()


@pytest.mark.parametrize("prec,learned_guess,form", [(0, False, {}), (1, False, {}), (2, False, {}), (2, True, {}),
                                                     (2, True, {"jvp_fp32": 1})])
def test_hex2048_three_steps_match_oracle(env, prec, learned_guess, form):
    """The 2048^2 precision workload (128 x 128 cores, 16,384 blocks), its first 3 steps; also the
    bench's headline form (FP32 JVP)."""
    P, torch, learned = env
    rec = G.load("hex2048_s3")
    s, net, w = _solver(P, torch, learned, "hex2048", prec, learned_guess, **form)
    s.set_field(w["phi"])
    infos = s.run(rec["meta"]["steps"])
    err, rel_e = check_against(rec, infos, s.get_field(), TOL["f64" if prec == 0 and not learned_guess else "mixed"])
    print(f"hex2048 prec {prec} learned {learned_guess} {form}: max|dphi| {err:.2e}, energy {rel_e:.2e}")
    s.close()
    if net is not None:
        net.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_bcc64_fifty_steps_match_oracle(env, prec):
    """The 3D BCC recipe on 64^3 (7 x 7 x 7 uneven cores, shifted ILU(0) blocks), all 50 adaptive steps."""
    P, torch, learned = env
    rec = G.load("bcc64_s50")
    s, _, w = _solver(P, torch, learned, "bcc64", prec)
    s.set_field(w["phi"])
    infos = s.run(rec["meta"]["steps"])
    err, rel_e = check_against(rec, infos, s.get_field(), TOL["f64" if prec == 0 else "mixed"])
    print(f"bcc64 prec {prec}: max|dphi| {err:.2e}, energy {rel_e:.2e}")
    s.close()


def test_ensemble_members_match_oracle(env):
    """The 32-run 256^2 ensemble stepped together by pfc_run_batch (BF16 factors, the bench's
    settings), 100 steps: members 3 and 22 against their oracle trajectories."""
    P, torch, learned = env
    w = inputs.workload("batch32x256")
    solvers = []
    for g in w["gammas"]:
        params = P.default_params(sub=tuple(w["parts"][::-1]), overlap=1, factor_prec=2, dt_min=w["dt_min"],
                                  dt_max=w["dt_max"], eta=w["eta"], gmres_max_it=1200, dt_halvings=6)
        solvers.append(P.Solver(w["shape"], w["h"], g, params, stream=torch.cuda.Stream()))
    for s, phi in zip(solvers, w["phis"]):
        s.set_field(phi)
    recs = P.run_batch(solvers, 100)
    for member in (3, 22):
        rec = G.load(f"batch{member}_s100")
        assert all(r["dt_cuts"] == 0 for r in recs[member])
        err, rel_e = check_against(rec, recs[member], solvers[member].get_field(), TOL["mixed"])
        print(f"ensemble member {member}: max|dphi| {err:.2e}, energy {rel_e:.2e}")
    for s in solvers:
        s.close()
