"""GPU tests of the batched runner pfc_run_batch (independent states on their
own streams stepped together by one captured graph per ensemble step) and of the
graph form of a time step: both give the same records and fields as the
host-driven steps, and each agrees with the oracle."""
import math

import numpy as np
import pytest

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H = math.pi / 4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P, torch


def _make(P, torch, shape, gamma, prec, stream=None):
    params = P.default_params(sub=(3, 3), overlap=1, factor_prec=prec, dt_min=0.01, dt_max=10.0, eta=5000.0)
    return P.Solver(shape, H, gamma, params, stream=stream)


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_equals_sequential_runs(env, prec):
    P, torch = env
    shape = (48, 48)
    gammas = [0.1, 0.18, 0.25, 0.33]
    phis = [inputs.noise_field(shape, 0.07, 0.07, 1004 + i) for i in range(4)]
    streams = [torch.cuda.Stream() for _ in gammas]
    batch = [_make(P, torch, shape, g, prec, st) for g, st in zip(gammas, streams)]
    for s, phi in zip(batch, phis):
        s.set_field(phi)
    g0 = P.launch_counts()["graphs"]
    recs = P.run_batch(batch, 3)
    torch.cuda.synchronize()
    assert P.launch_counts()["graphs"] - g0 == 1  # step 1 tunes on threads; steps 2-3: one graph launch
    for i, (g, phi) in enumerate(zip(gammas, phis)):
        s = _make(P, torch, shape, g, prec)
        s.set_field(phi)
        ref = s.run(3)
        assert [r["newton_its"] for r in recs[i]] == [r["newton_its"] for r in ref]
        assert [r["dt"] for r in recs[i]] == [r["dt"] for r in ref]
        np.testing.assert_array_equal(batch[i].get_field(), s.get_field())


def test_batch_member_matches_oracle(env):
    """One member of a batch (gamma 0.18) against the oracle's adaptive run."""
    P, torch = env
    shape = (48, 48)
    gammas = [0.3, 0.18]
    phis = [inputs.noise_field(shape, 0.07, 0.07, 1010 + i) for i in range(2)]
    batch = [_make(P, torch, shape, g, 0, torch.cuda.Stream()) for g in gammas]
    for s, phi in zip(batch, phis):
        s.set_field(phi)
    recs = P.run_batch(batch, 3)
    ref, orecs = O.run(phis[1], H, gammas[1], O.Params(parts=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0,
                                                       eta=5000.0), 3)
    assert np.abs(batch[1].get_field() - ref).max() <= 1e-8
    for r, o in zip(recs[1], orecs):
        assert abs(r["energy"] - o.energy) <= 1e-10 * abs(o.energy)


def test_batch_rejects_bad_arguments(env):
    P, torch = env
    with pytest.raises(P.PfcError):
        P.run_batch([], 1)


def test_failed_steps_are_retried_with_half_the_step(env):
    """With GMRES capped at 8 iterations the larger controller steps fail; pfc_run
    halves dt (dt_halvings) until the step converges, and the accepted phi^{n+1}
    satisfies the scheme at the dt actually used (oracle residual)."""
    P, torch = env
    shape = (48, 48)
    params = P.default_params(sub=(3, 3), overlap=1, factor_prec=0, dt_min=0.01, dt_max=10.0, eta=5000.0,
                              gmres_max_it=8, dt_halvings=12)
    s = P.Solver(shape, H, 0.33, params)
    phi = inputs.noise_field(shape, 0.07, 0.07, 1020)
    s.set_field(phi)
    prev = phi
    cuts = 0
    for _ in range(4):
        rec = s.run(1)[0]
        cur = s.get_field()
        cuts += rec["dt_cuts"]
        r_new = np.linalg.norm(O.residual(cur, prev, rec["dt"], H, 0.33))
        r_ref = np.linalg.norm(O.residual(prev, prev, rec["dt"], H, 0.33))
        assert r_new <= 1e-10 * r_ref * 1.01
        prev = cur
    assert cuts > 0
    s0 = P.Solver(shape, H, 0.33, P.default_params(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0,
                                                   gmres_max_it=8))
    s0.set_field(phi)
    with pytest.raises(P.PfcError) as e:
        s0.run(4)
    assert e.value.status == P.PFC_EGMRES


def _graph_vs_host(P, torch, shape, sub, prec, steps, phi, gamma=0.25, fixed_dt=None, **kw):
    """Both forms over `steps` steps (adaptive dt, or fixed_dt); with apply_variant = -1 the first
    step tunes the apply kernel on the host, every later step is one graph launch."""
    out = {}
    for ug in (0, 1):
        params = P.default_params(sub=sub, overlap=1, factor_prec=prec, dt_min=0.01, dt_max=10.0, eta=5000.0,
                                  use_graph=ug, **kw)
        s = P.Solver(shape, H, gamma, params, stream=torch.cuda.Stream())
        s.set_field(phi)
        g0 = P.launch_counts()["graphs"]
        recs = [s.step(fixed_dt) for _ in range(steps)] if fixed_dt else s.run(steps)
        out[ug] = (recs, s.get_field(), s.tuning()["graph"], P.launch_counts()["graphs"] - g0)
        s.close()
    tuned_first = kw.get("apply_variant", -1) < 0
    assert out[1][2] == 1 and out[0][2] == 0
    assert out[1][3] == steps - tuned_first and out[0][3] == 0  # one graph per step
    for key in ("newton_its", "gmres_its", "ls_cuts", "dt", "energy", "res_norm"):
        assert [r[key] for r in out[0][0]] == [r[key] for r in out[1][0]], key
    np.testing.assert_array_equal(out[0][1], out[1][1])
    return out


@pytest.mark.parametrize("prec", [0, 2])
def test_graph_steps_match_the_host_loop(env, prec):
    """Whole time steps captured as CUDA graphs (use_graph = 1: Newton loop, factor branch,
    GMRES restart and Arnoldi loops, line search and commit as conditional nodes driven by
    device-side control kernels) run the same kernels in the same order as the host-driven
    step: identical records and fields, bit for bit."""
    P, torch = env
    shape = (64, 64)
    out = _graph_vs_host(P, torch, shape, (4, 4), prec, 4, inputs.noise_field(shape, 0.07, 0.07, 1030))
    assert sum(r["gmres_its"] for r in out[1][0]) > 60  # GMRES(30) restarted within some Newton iterations


def test_graph_steps_match_the_host_loop_at_512(env):
    """The same at 512^2 (256 tiles per vector in the Gram-Schmidt sweeps, more than the CTAs of a
    sweep), BF16 factors, 3 steps: the host loop sizes its sweeps like the graph's."""
    P, torch = env
    shape = (512, 512)
    _graph_vs_host(P, torch, shape, (32, 32), 2, 3, inputs.hex_seeds_2d(shape, H, seed=2100))


def test_graph_steps_with_line_search_cuts_match_the_host_loop(env):
    """Variable mobility at dt = 10 from a crystal seed needs damped Newton steps: the
    device-side line search (Armijo test, quadratic backtracking) takes the same cuts in both
    forms.  A fixed apply kernel makes every step of the graph form a graph launch."""
    P, torch = env
    shape = (48, 48)
    phi = inputs.hex_seeds_2d(shape, H, nseeds=1, radius_cells=10, seed=3)
    out = _graph_vs_host(P, torch, shape, (3, 3), 1, 2, phi, fixed_dt=10.0, mobility=1, apply_variant=5)
    assert sum(r["ls_cuts"] for r in out[1][0]) > 0


def test_batch_time_loop_retries_like_pfc_run(env):
    """States whose steps fail (GMRES capped at 8 iterations) retry with dt / 2 inside the batch
    graph's device time loop exactly as pfc_run retries them on the host: the same records
    (dt, halvings, iterations) and bit-identical fields."""
    P, torch = env
    shape = (48, 48)
    gammas = [0.2, 0.33, 0.28]
    phis = [inputs.noise_field(shape, 0.07, 0.07, 1050 + i) for i in range(3)]

    def make(g, st):
        prm = P.default_params(sub=(3, 3), overlap=1, dt_min=0.01, dt_max=10.0, eta=5000.0, gmres_max_it=8,
                               dt_halvings=12)
        return P.Solver(shape, H, g, prm, stream=st)

    batch = [make(g, torch.cuda.Stream()) for g in gammas]
    for s, phi in zip(batch, phis):
        s.set_field(phi)
    g0 = P.launch_counts()["graphs"]
    recs = P.run_batch(batch, 5)
    assert P.launch_counts()["graphs"] - g0 == 1  # steps 2-5 of every state in one graph launch
    assert sum(r["dt_cuts"] for rr in recs for r in rr[1:]) > 0
    for i, (g, phi) in enumerate(zip(gammas, phis)):
        s = make(g, None)
        s.set_field(phi)
        ref = s.run(5)
        for key in ("dt", "dt_cuts", "newton_its", "gmres_its", "energy"):
            assert [r[key] for r in recs[i]] == [r[key] for r in ref], (i, key)
        np.testing.assert_array_equal(batch[i].get_field(), s.get_field())
