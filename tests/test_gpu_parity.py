"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.  Tolerances: FP64 kernels to rounding (1e-12 relative
for single operators); full steps to max|phi_gpu - phi_oracle| <= 1e-8 and
relative energy error <= 1e-10 (plain FP64 path)."""
import math

import numpy as np
import pytest

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H = math.pi / 4
GAMMA = 0.25


@pytest.fixture(scope="module")
def pfc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P


def solver(P, shape, parts, prec=0, **kw):
    params = P.default_params(sub=tuple(parts[::-1]), factor_prec=prec, **kw)
    return P.Solver(shape, H, GAMMA, params)


@pytest.mark.parametrize("shape", [(64, 64), (40, 70), (9, 13), (48, 200)])
def test_residual_matches_oracle(pfc, shape):
    Phi = inputs.noise_field(shape, 0.2, 0.4, 1)
    phin = inputs.noise_field(shape, 0.2, 0.4, 2)
    s = solver(pfc, shape, (1, 1), overlap=0)
    F, nrm = s.residual(Phi, phin, 0.7)
    ref = O.residual(Phi, phin, 0.7, H, GAMMA)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * scale)
    assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)


@pytest.mark.parametrize("shape", [(64, 64), (40, 70), (33, 31), (96, 130)])
def test_fp32_jvp_matches_oracle(pfc, shape):
    """The opt-in plain FP32 JVP of the mixed path (jvp_fp32 = 1): inputs cut to floats and an
    FP32 stencil whose terms reach ih2^3 |v| ~ 4 |v| times 20 in the radius-3 sum, so each entry
    is within about 2^-24 x 100 of max |J v|; the bound asserted is 1e-5 of the largest entry."""
    Phi = inputs.noise_field(shape, 0.2, 0.4, 3)
    phin = inputs.noise_field(shape, 0.2, 0.4, 4)
    v = inputs.noise_field(shape, 0.0, 1.0, 5)
    s = solver(pfc, shape, (1, 1), prec=2, overlap=0, jvp_fp32=1)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 2.5, H, GAMMA)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    assert np.abs(Jv - ref).max() > 1e-12 * np.abs(ref).max()  # it is the FP32 kernel, not the float-float one


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("shape", [(64, 64), (40, 70), (33, 31), (96, 130), (80, 200)])
def test_jvp_matches_oracle(pfc, shape, prec):
    """FP64 JVP (plain path) and the float-float JVP of the mixed path (F32/BF16
    factors): both within 1e-12 of the oracle, relative to the largest entry.  On the mixed
    path the 96 x 130 and 80 x 200 grids have interior tiles, whose halos come by TMA tensor
    copies, beside edge tiles staged by plain loads."""
    Phi = inputs.noise_field(shape, 0.2, 0.4, 3)
    phin = inputs.noise_field(shape, 0.2, 0.4, 4)
    v = inputs.noise_field(shape, 0.0, 1.0, 5)
    s = solver(pfc, shape, (1, 1), prec=prec, overlap=0)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 2.5, H, GAMMA)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_float_float_jvp_on_a_smooth_vector(pfc):
    """A smooth v makes the stencil terms cancel (J v ~ v / dt at dt = 10 while the
    Delta_d^3 terms are ~ 1e2 |v|): the float-float JVP must still agree with the
    oracle to 1e-11 of max |J v|."""
    shape = (64, 64)
    Phi = inputs.noise_field(shape, 0.2, 0.4, 3)
    phin = inputs.noise_field(shape, 0.2, 0.4, 4)
    v = inputs.sine_field(shape, H, 1.0, 32.0 * H)
    s = solver(pfc, shape, (1, 1), prec=2, overlap=0)
    Jv = s.jvp(Phi, phin, v, 10.0).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 10.0, H, GAMMA)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(64, 64), (37, 50)])
def test_energy_mass_match_oracle(pfc, shape):
    phi = inputs.hex_seeds_2d(shape, H, nseeds=1, radius_cells=6, seed=7) if shape == (64, 64) else \
        inputs.noise_field(shape, 0.1, 0.3, 6)
    s = solver(pfc, shape, (1, 1), overlap=0)
    s.set_field(phi)
    assert s.energy() == pytest.approx(O.energy(phi, H, GAMMA), rel=1e-12)
    assert s.mass() == pytest.approx(O.mass(phi, H), rel=1e-12, abs=1e-12)


# F64 factors: the same LU as the oracle's up to rounding.  F32 / BF16 storage
# (unit roundoff 2^-24 / 2^-9 per factor entry) perturbs the banded solves by
# that roundoff times the growth of the triangular factors; at dt = 10 the
# blocks are near-indefinite and BF16 storage reaches ~0.1 relative.  An
# error of order one would mean a wrong factor, not storage rounding.
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 0.25)])
@pytest.mark.parametrize("shape,parts,dt", [((64, 64), (4, 4), 0.1), ((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0)])
def test_precond_apply_matches_oracle(pfc, shape, parts, dt, prec, tol):
    """Left-RAS with the improved-BC block factors (Eqs. ras, Ak) against the
    oracle's dense-LU Schwarz apply; F32/BF16 factor storage within their rounding."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=prec, overlap=1)
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, dt, H, GAMMA)
    pre = O.Schwarz(J, O.decompose(shape, parts, 1), "left-ras", "lu")
    ref = pre.apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("shape,parts,dt", [((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0)])
def test_apply_launch_shapes_agree(pfc, shape, parts, dt, prec):
    """Every apply launch shape (chunk length, warps per CTA, one or two subdomains
    per warp) runs the same eliminations in the same order: identical results on
    ragged decompositions (four block extents, so the two-per-warp order carries
    padding slots)."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    z = {}
    for v in (0, 1, 2, 3, 4):
        s = solver(pfc, shape, parts, prec=prec, overlap=1, apply_variant=v)
        z[v] = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
        assert s.tuning()["apply_variant"] == v
    for v in (1, 2, 3, 4):
        np.testing.assert_array_equal(z[v], z[0])


def test_apply_autotuner_picks_a_timed_kernel(pfc):
    """apply_variant = -1 times every kernel that fits at the first factorisation
    and keeps the fastest; the step result does not depend on the pick."""
    w = inputs.workload("noise64")
    out = {}
    for v in (-1, 0):
        s = solver(pfc, w["shape"], w["parts"], prec=2, overlap=1, apply_variant=v)
        s.set_field(w["phi"])
        for _ in range(2):
            s.step(w["fixed_dt"])
        out[v] = s.get_field()
        t = s.tuning()
        if v == -1:
            assert t["apply_variant"] in range(pfc.N_APPLY_VARIANTS)
            assert all(ms > 0 for ms in t["apply_ms"])
            # the fastest shape, or a lower-numbered one within 1 % of it
            assert t["apply_ms"][t["apply_variant"]] <= 1.01 * min(t["apply_ms"])
            assert all(ms > 1.01 * min(t["apply_ms"]) for ms in t["apply_ms"][:t["apply_variant"]])
        else:
            assert t["apply_ms"] == [-1.0] * pfc.N_APPLY_VARIANTS
    assert np.abs(out[-1] - out[0]).max() <= 1e-9


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4)])
def test_wide_blocks_use_the_wide_window_kernel(pfc, prec, tol):
    """24-cell-wide blocks (kl = 72 > 64) run the wide-window apply kernel or the
    chunked one: same oracle parity; the other launch shapes are refused."""
    shape = (44, 44)
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    J = O.assemble_jacobian(Phi, phin, 1.0, H, GAMMA)
    ref = O.Schwarz(J, O.decompose(shape, (2, 2), 1), "left-ras", "lu").apply(r)
    for v in (-1, 0, pfc.APPLY_CHUNKED):
        s = solver(pfc, shape, (2, 2), prec=prec, overlap=1, apply_variant=v)
        z = s.precond_apply(Phi, phin, 1.0, r).cpu().numpy()
        assert s.tuning()["apply_variant"] in (0, pfc.APPLY_CHUNKED)
        assert np.linalg.norm(z - ref) / np.linalg.norm(ref) <= tol
    s2 = solver(pfc, shape, (2, 2), prec=prec, overlap=1, apply_variant=1)
    with pytest.raises(pfc.PfcError) as e:
        s2.precond_apply(Phi, phin, 1.0, r)
    assert e.value.status == pfc.PFC_EINVAL


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 0.25)])
@pytest.mark.parametrize("shape,parts,dt", [((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0),
                                            ((21, 27), (3, 3), 10.0)])
def test_chunked_apply_matches_oracle(pfc, shape, parts, dt, prec, tol):
    """The chunked solves (apply variant 5: the factors regrouped 8 elimination
    steps at a time, a row permutation and an 8-column product per group) against
    the oracle's dense-LU Schwarz apply, on ragged decompositions (block sizes
    360 ... 399 and 315 ... 352 cells, most with a partial last chunk, and 99)."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=prec, overlap=1, apply_variant=pfc.APPLY_CHUNKED)
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    assert s.tuning()["apply_variant"] == pfc.APPLY_CHUNKED
    J = O.assemble_jacobian(Phi, phin, dt, H, GAMMA)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1), "left-ras", "lu").apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err
    if prec == 0:  # the per-step solves on the same FP64 factors agree to rounding
        s0 = solver(pfc, shape, parts, prec=0, overlap=1, apply_variant=0)
        z0 = s0.precond_apply(Phi, phin, dt, r).cpu().numpy()
        assert np.abs(z - z0).max() <= 1e-12 * np.abs(z0).max()


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (2, 1e-7)])
def test_chunked_apply_steps_match_oracle(pfc, prec, tol):
    """Five adaptive steps of the 64^2 noise field with the chunked apply: the
    Newton solutions against the oracle's (the preconditioner only changes the
    path, not the discrete solution)."""
    w = inputs.workload("noise64")
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, w["shape"], w["parts"], prec=prec, overlap=1, apply_variant=pfc.APPLY_CHUNKED, **prm)
    s.set_field(w["phi"])
    recs = s.run(5)
    ref, orecs = O.run(w["phi"], w["h"], w["gamma"], O.Params(parts=w["parts"], overlap=1, **prm), 5)
    assert np.abs(s.get_field() - ref).max() <= tol
    assert [r["dt"] for r in recs] == pytest.approx([o.dt for o in orecs], rel=1e-9)


KINDS = {"as": 0, "right-ras": 2, "left-ras": 1}  # oracle name -> PFC_AS / PFC_RIGHT_RAS / PFC_LEFT_RAS


@pytest.mark.parametrize("kind", ["as", "right-ras"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 0.25)])
@pytest.mark.parametrize("shape,parts,dt", [((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0)])
def test_schwarz_kinds_match_oracle(pfc, shape, parts, dt, prec, tol, kind):
    """Additive Schwarz (Eq. invM: solve on the overlapped block, add every block's whole
    solution) and right-RAS (Eq. ash: the core of r in, the whole block out) against the
    oracle's dense-LU forms, on ragged decompositions (overlap sums of 2 and 4 blocks)."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=prec, overlap=1, ras_kind=KINDS[kind])
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, dt, H, GAMMA)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1), kind, "lu").apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("kind", ["left-ras", "as", "right-ras"])
@pytest.mark.parametrize("overlap", [0, 2, 3])
def test_overlaps_match_oracle(pfc, kind, overlap):
    """Overlaps of 0, 2 and 3 cells per side (blocks of 16, 20 and 22 cells: the last runs
    kl = 66, past the narrow kernels) for the three Schwarz forms, FP64 factors."""
    shape, parts = (96, 80), (5, 6)
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=0, overlap=overlap, ras_kind=KINDS[kind])
    z = s.precond_apply(Phi, phin, 10.0, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, 10.0, H, GAMMA)
    ref = O.Schwarz(J, O.decompose(shape, parts, overlap), kind, "lu").apply(r)
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) <= 1e-11


@pytest.mark.parametrize("kind", ["as", "right-ras"])
def test_schwarz_kinds_steps_match_oracle(pfc, kind):
    """Two adaptive steps of the 48^2 noise field with AS and right-RAS, FP64 factors:
    the Newton solutions against the oracle's with the same preconditioner."""
    shape = (48, 48)
    phi = inputs.noise_field(shape, 0.07, 0.07, 1050)
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, shape, (3, 3), prec=0, overlap=1, ras_kind=KINDS[kind], **prm)
    s.set_field(phi)
    s.run(2)
    ref, _ = O.run(phi, H, GAMMA, O.Params(parts=(3, 3), overlap=1, ras_kind=kind, **prm), 2)
    assert np.abs(s.get_field() - ref).max() <= 1e-8


@pytest.mark.parametrize("shape", [(64, 64), (40, 70), (48, 200)])
def test_mobility_operators_match_oracle(pfc, shape):
    """Variable mobility M = 1 - phi^2 (Sec. 3, Eq. NSOP): residual and JVP (with the dM/dPhi
    term) against the oracle."""
    Phi = inputs.noise_field(shape, 0.2, 0.4, 1)
    phin = inputs.noise_field(shape, 0.2, 0.4, 2)
    v = inputs.noise_field(shape, 0.0, 1.0, 3)
    s = solver(pfc, shape, (2, 2), overlap=1, mobility=1)
    F, nrm = s.residual(Phi, phin, 0.7)
    ref = O.residual(Phi, phin, 0.7, H, GAMMA, mobility=True)
    assert np.abs(F.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    Jv = s.jvp(Phi, phin, v, 0.7).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 0.7, H, GAMMA, mobility=True)
    assert np.abs(Jv - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [(0, 5e-11), (1, 2e-2)])
@pytest.mark.parametrize("shape,parts,dt", [((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0)])
def test_mobility_precond_matches_oracle(pfc, shape, parts, dt, prec, tol):
    """Left-RAS on the mobility Jacobian: the block matrices (principal submatrices, with the
    edge mobilities and the dM/dPhi coupling) against the oracle's dense-LU Schwarz apply.
    Two backward-stable LU solves differ by about cond(A_k) eps: on this noise field at dt = 10
    cond(A_k) is near 1e5 (FP64: 1e-11 measured; F32 storage: 7e-3), so the F32 bound is loose
    and the FP64 case carries the check of every entry."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=prec, overlap=1, mobility=1)
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, dt, H, GAMMA, mobility=True)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1), "left-ras", "lu").apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (2, 1e-7)])
def test_mobility_steps_match_oracle(pfc, prec, tol):
    """Three adaptive steps of a 48^2 noise field with M = 1 - phi^2 against the oracle; mass
    conserved and energy non-increasing on the way."""
    shape = (48, 48)
    phi = inputs.noise_field(shape, 0.07, 0.07, 1060)
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, shape, (3, 3), prec=prec, overlap=1, mobility=1, **prm)
    s.set_field(phi)
    recs = s.run(3)
    ref, orecs = O.run(phi, H, GAMMA, O.Params(parts=(3, 3), overlap=1, mobility=True, **prm), 3)
    assert np.abs(s.get_field() - ref).max() <= tol
    for r, o in zip(recs, orecs):
        assert abs(r["energy"] - o.energy) <= 1e-9 * abs(o.energy)
    assert all(b["energy"] <= a["energy"] + 1e-13 * abs(a["energy"]) for a, b in zip(recs, recs[1:]))


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (2, 1e-7)])
def test_factor_reuse_across_steps_keeps_the_solution(pfc, prec, tol):
    """reuse_factor = 3: the subdomain factors of one step serve up to three more steps at the
    same dt (the controller holds dt = dt_max on this field after its first steps); the
    Newton solutions still match the oracle, which refactors every step."""
    w = inputs.workload("noise64")
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, w["shape"], w["parts"], prec=prec, overlap=1, reuse_factor=3, **prm)
    s.set_field(w["phi"])
    recs = s.run(6)
    ref, orecs = O.run(w["phi"], w["h"], w["gamma"], O.Params(parts=w["parts"], overlap=1, **prm), 6)
    assert np.abs(s.get_field() - ref).max() <= tol
    assert [r["dt"] for r in recs] == pytest.approx([o.dt for o in orecs], rel=1e-9)


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (2, 1e-7)])
@pytest.mark.parametrize("shape", [(27, 21), (45, 37)])
def test_odd_point_count_steps_match_oracle(pfc, shape, prec, tol):
    """Grids of 567 and 1665 points: every Krylov vector has odd length, so the last
    tile of each streamed Gram-Schmidt sweep is partial and odd (1665 = 1024 + 641);
    two adaptive steps against the oracle's."""
    phi = inputs.noise_field(shape, 0.07, 0.07, 1040)
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, shape, (3, 3), prec=prec, overlap=1, **prm)
    s.set_field(phi)
    s.run(2)
    ref, _ = O.run(phi, H, GAMMA, O.Params(parts=(3, 3), overlap=1, **prm), 2)
    assert np.abs(s.get_field() - ref).max() <= tol


def test_twenty_steps_noise64_match_oracle(pfc):
    """64^2 liquid from noise, fixed dt = 0.1, 20 steps, left-RAS 4x4 cores of 16^2 with
    one overlap cell per side (18^2 blocks): phi and energy per step against the oracle."""
    w = inputs.workload("noise64")
    s = solver(pfc, w["shape"], w["parts"], overlap=1)
    s.set_field(w["phi"])
    infos = [s.step(w["fixed_dt"]) for _ in range(w["steps"])]
    got = s.get_field()
    ref, recs = O.run(w["phi"], w["h"], w["gamma"], O.Params(parts=w["parts"], overlap=1), w["steps"],
                      fixed_dt=w["fixed_dt"])
    assert np.abs(got - ref).max() <= 1e-8
    for inf, rec in zip(infos, recs):
        assert abs(inf["energy"] - rec.energy) <= 1e-10 * abs(rec.energy)
        assert abs(inf["mass"] - rec.mass) <= 1e-12 * max(1.0, abs(rec.mass))
    E = [i["energy"] for i in infos]
    assert all(b <= a for a, b in zip(E, E[1:]))


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_factors_match_oracle(pfc, prec):
    """F32 / BF16 factor storage changes only the preconditioner: the Newton
    solution stays within 1e-7 (phi) and 1e-9 (relative energy) of the FP64 oracle."""
    w = inputs.workload("noise64")
    s = solver(pfc, w["shape"], w["parts"], prec=prec, overlap=1)
    s.set_field(w["phi"])
    infos = [s.step(w["fixed_dt"]) for _ in range(5)]
    ref, recs = O.run(w["phi"], w["h"], w["gamma"], O.Params(parts=w["parts"], overlap=1), 5, fixed_dt=w["fixed_dt"])
    assert np.abs(s.get_field() - ref).max() <= 1e-7
    assert abs(infos[-1]["energy"] - recs[-1].energy) <= 1e-9 * abs(recs[-1].energy)


def test_adaptive_run_matches_oracle(pfc):
    """pfc_run with the adaptive step (Eq. sencondt) on a small crystal-growth
    case (ragged 3x2 decomposition) against the oracle's time loop."""
    shape = (48, 60)
    phi0 = inputs.hex_seeds_2d(shape, H, nseeds=1, radius_cells=8, seed=11)
    prm = dict(dt_min=0.01, dt_max=10.0, eta=5000.0)
    s = solver(pfc, shape, (3, 2), overlap=1, **prm)
    s.set_field(phi0)
    infos = s.run(12)
    ref, recs = O.run(phi0, H, GAMMA, O.Params(parts=(3, 2), overlap=1, **prm), 12)
    for inf, rec in zip(infos, recs):
        assert inf["dt"] == pytest.approx(rec.dt, rel=1e-8)
        assert abs(inf["energy"] - rec.energy) <= 1e-10 * abs(rec.energy)
    assert np.abs(s.get_field() - ref).max() <= 1e-8


def test_constant_field_takes_no_newton_iteration(pfc):
    shape = (32, 32)
    s = solver(pfc, shape, (2, 2), overlap=1)
    s.set_field(np.full(shape, 0.3))
    info = s.step(1.0)
    assert info["newton_its"] == 0 and np.array_equal(s.get_field(), np.full(shape, 0.3))


def test_invalid_arguments_and_small_workspace(pfc):
    import ctypes

    s = solver(pfc, (32, 32), (2, 2), overlap=1)
    with pytest.raises(pfc.PfcError) as e:
        s.step(-1.0)
    assert e.value.status == pfc.PFC_EINVAL
    g = pfc.make_grid((32, 32))
    p = pfc.default_params(sub=(2, 2))
    h = ctypes.c_void_p()
    st = pfc.lib().pfc_create(ctypes.byref(g), H, GAMMA, ctypes.byref(p), ctypes.c_void_p(s.ws.data_ptr()),
                              ctypes.c_size_t(1024), None, ctypes.byref(h))
    assert st == pfc.PFC_ENOMEM


def test_checkpoint_resume_continues_the_same_run(pfc, tmp_path):
    """pfc_save after 3 adaptive steps, pfc_load into a fresh state: the next 2
    steps equal those of the uninterrupted run (fields bitwise, same dt); a state
    of another grid refuses the file."""
    shape = (48, 60)
    phi0 = inputs.hex_seeds_2d(shape, H, nseeds=1, radius_cells=8, seed=11)
    prm = dict(dt_min=0.01, dt_max=10.0, eta=5000.0)
    a = solver(pfc, shape, (3, 2), overlap=1, **prm)
    a.set_field(phi0)
    a.run(3)
    path = str(tmp_path / "state.pfc")
    a.save(path)
    ra = a.run(2)
    b = solver(pfc, shape, (3, 2), overlap=1, **prm)
    b.load(path)
    rb = b.run(2)
    assert [r["dt"] for r in ra] == [r["dt"] for r in rb]
    np.testing.assert_array_equal(a.get_field(), b.get_field())
    c = solver(pfc, (48, 48), (3, 3), overlap=1, **prm)
    with pytest.raises(pfc.PfcError) as e:
        c.load(path)
    assert e.value.status == pfc.PFC_EINVAL


# ---------------------------------------------------------------- Neumann-type walls (Sec. 2)
NEU = 1  # PFC_NEUMANN


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("shape", [(64, 64), (40, 70), (9, 13), (48, 200)])
def test_neumann_operators_match_oracle(pfc, shape, prec):
    """Mirror walls: residual, J v (FP64 and float-float), energy and mass against the oracle's
    even-extension operators; the fields differ most near the walls, where the stencils fold."""
    Phi = inputs.noise_field(shape, 0.2, 0.4, 1)
    phin = inputs.noise_field(shape, 0.2, 0.4, 2)
    v = inputs.noise_field(shape, 0.0, 1.0, 3)
    s = solver(pfc, shape, (1, 1), prec=prec, overlap=0, boundary=NEU)
    F, nrm = s.residual(Phi, phin, 0.7)
    ref = O.residual(Phi, phin, 0.7, H, GAMMA, neumann=True)
    np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 2.5, H, GAMMA, neumann=True)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    s.set_field(Phi)
    assert s.energy() == pytest.approx(O.energy(Phi, H, GAMMA, neumann=True), rel=1e-12)
    assert s.mass() == pytest.approx(O.mass(Phi, H), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("variant", [0, 4, 5])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 0.25)])
@pytest.mark.parametrize("shape,parts,dt", [((50, 37), (3, 2), 10.0), ((96, 80), (5, 6), 1.0),
                                            ((21, 27), (3, 3), 10.0)])
def test_neumann_precond_matches_oracle(pfc, shape, parts, dt, prec, tol, variant):
    """Left-RAS between mirror walls: the wall blocks are clipped (no wrap) and their matrices
    carry the folded mirror entries; per-step and chunked solves against the oracle's dense-LU
    Schwarz apply, with the periodic tests' rounding bounds."""
    Phi = inputs.noise_field(shape, 0.285, 0.3, 8)
    phin = inputs.noise_field(shape, 0.285, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver(pfc, shape, parts, prec=prec, overlap=1, apply_variant=variant, boundary=NEU)
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, dt, H, GAMMA, neumann=True)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1, neumann=True), "left-ras", "lu").apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (2, 1e-7)])
def test_neumann_steps_match_oracle(pfc, prec, tol):
    """Three adaptive steps of a 48 x 40 noise field between mirror walls against the oracle;
    mass conserved and the energy non-increasing."""
    shape = (48, 40)
    phi = inputs.noise_field(shape, 0.07, 0.07, 1070)
    prm = dict(dt_min=1e-2, dt_max=10.0, eta=5000.0)
    s = solver(pfc, shape, (3, 3), prec=prec, overlap=1, boundary=NEU, **prm)
    s.set_field(phi)
    recs = s.run(3)
    ref, orecs = O.run(phi, H, GAMMA, O.Params(parts=(3, 3), overlap=1, neumann=True, **prm), 3)
    assert np.abs(s.get_field() - ref).max() <= tol
    for r, o in zip(recs, orecs):
        assert abs(r["energy"] - o.energy) <= 1e-9 * abs(o.energy)
        assert abs(r["mass"] - o.mass) <= 1e-12 * max(1.0, abs(o.mass))
    assert all(b["energy"] <= a["energy"] + 1e-13 * abs(a["energy"]) for a, b in zip(recs, recs[1:]))


# ---------------------------------------------------------------- crack propagation (Test C)
@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 1e-7)])
def test_crack_steps_match_oracle(pfc, prec, tol):
    """Test C's recipe (stretched lattice, liquid notch of 40 x 20 cells, gamma = 1, dt in [1, 5],
    eta = 100) on a 128 x 48 grid: three adaptive steps against the oracle, the second one a hard
    step (11 Newton iterations, line-search cuts, thousands of GMRES iterations in the oracle).
    Tightening the oracle's tolerances moves its solution by 2e-12, loosening GMRES to 1e-3 by 2e-9."""
    w = inputs.workload("crack128x48")
    prm = dict(dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"])
    params = pfc.default_params(sub=tuple(w["parts"][::-1]), factor_prec=prec, overlap=1, **prm)
    s = pfc.Solver(w["shape"], w["h"], w["gamma"], params)
    s.set_field(w["phi"])
    recs = s.run(3)
    ref, orecs = O.run(w["phi"], w["h"], w["gamma"], O.Params(parts=w["parts"], overlap=1, **prm), 3)
    assert np.abs(s.get_field() - ref).max() <= tol
    assert [r["dt"] for r in recs] == pytest.approx([o.dt for o in orecs], rel=1e-9)
    for r, o in zip(recs, orecs):
        assert abs(r["energy"] - o.energy) <= 1e-9 * abs(o.energy)
