"""GPU parity of the 3D path (7-point Laplacian, 63-point composed operators,
level-scheduled shifted ILU(0) Schwarz blocks) against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

pytestmark = pytest.mark.gpu

H3 = 80 * math.pi / 256
GAMMA3 = 0.3


@pytest.fixture(scope="module")
def pfc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P


def solver3(P, shape, parts, prec=0, **kw):
    params = P.default_params(sub=tuple(parts[::-1]), factor_prec=prec, overlap=1, **kw)
    return P.Solver(shape, H3, GAMMA3, params)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 14, 18)])
def test_residual_jvp_energy_3d(pfc, shape):
    Phi = inputs.noise_field(shape, -0.3, 0.4, 1)
    phin = inputs.noise_field(shape, -0.3, 0.4, 2)
    v = inputs.noise_field(shape, 0.0, 1.0, 3)
    s = solver3(pfc, shape, (2, 2, 2))
    F, nrm = s.residual(Phi, phin, 0.7)
    ref = O.residual(Phi, phin, 0.7, H3, GAMMA3)
    np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    refj = O.jvp(v, Phi, phin, 2.5, H3, GAMMA3)
    np.testing.assert_allclose(Jv, refj, rtol=0, atol=1e-12 * np.abs(refj).max())
    s.set_field(Phi)
    assert s.energy() == pytest.approx(O.energy(Phi, H3, GAMMA3), rel=1e-12)
    assert s.mass() == pytest.approx(O.mass(Phi, H3), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-4), (2, 0.05)])
@pytest.mark.parametrize("shape,parts,dt", [((16, 16, 16), (2, 2, 2), 2.0), ((17, 16, 15), (2, 2, 2), 0.5)])
def test_precond_apply_3d(pfc, shape, parts, dt, prec, tol):
    """Left-RAS with level-scheduled shifted ILU(0) blocks (uneven splits) against
    the oracle's ILU(0) of A_k + 0.1 mean|diag A_k| I."""
    Phi = inputs.noise_field(shape, -0.325, 0.3, 8)
    phin = inputs.noise_field(shape, -0.325, 0.3, 9)
    r = inputs.noise_field(shape, 0.0, 1.0, 10)
    s = solver3(pfc, shape, parts, prec=prec)
    z = s.precond_apply(Phi, phin, dt, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, dt, H3, GAMMA3)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1), "left-ras", "ilu0", 0.1).apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol_phi,tol_e", [(0, 1e-8, 1e-10), (2, 1e-7, 1e-9)])
def test_steps_3d_match_oracle(pfc, prec, tol_phi, tol_e):
    """Three fixed steps at dt = 0.5 on a 16^3 BCC-seeded field, 2x2x2 blocks: the plain FP64
    path, and the mixed path (BF16 factors in the level-window apply, float-float JVP) at the
    mixed tolerances."""
    shape = (16, 16, 16)
    phi0 = inputs.bcc_seeds_3d(shape, H3, nseeds=1, d0=4 * H3, seed=5)
    s = solver3(pfc, shape, (2, 2, 2), prec=prec)
    s.set_field(phi0)
    infos = [s.step(0.5) for _ in range(3)]
    ref, recs = O.run(phi0, H3, GAMMA3, O.Params(parts=(2, 2, 2), overlap=1, subdomain_solver="ilu0"), 3,
                      fixed_dt=0.5)
    assert np.abs(s.get_field() - ref).max() <= tol_phi
    for inf, rec in zip(infos, recs):
        assert abs(inf["energy"] - rec.energy) <= tol_e * abs(rec.energy)
    E = [i["energy"] for i in infos]
    assert all(b <= a for a, b in zip(E, E[1:]))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape,parts", [((74, 74, 74), (2, 2, 2)), ((80, 80, 80), (2, 2, 2)),
                                         ((17, 16, 15), (2, 2, 2)), ((36, 30, 27), (3, 2, 2))])
def test_window_apply_equals_global_apply(pfc, shape, parts, prec):
    """The shared-memory level-window apply (variant 1) and the global-memory apply (variant 0)
    take the same operations in the same order: bitwise equal outputs, on 39^3 blocks (the 256^3
    workload's, 218-row levels), 42^3 blocks (252-row levels, near the window's 255) and small
    and uneven ones."""
    Phi = inputs.noise_field(shape, -0.325, 0.3, 21)
    phin = inputs.noise_field(shape, -0.325, 0.3, 22)
    r = inputs.noise_field(shape, 0.0, 1.0, 23)
    sw = solver3(pfc, shape, parts, prec=prec, apply_variant=1)
    sg = solver3(pfc, shape, parts, prec=prec, apply_variant=0)
    assert sw.tuning()["apply_variant"] == 1 and sg.tuning()["apply_variant"] == 0
    assert solver3(pfc, shape, parts, prec=prec).tuning()["apply_variant"] == 1  # the default where it fits
    zw = sw.precond_apply(Phi, phin, 1.5, r).cpu().numpy()
    zg = sg.precond_apply(Phi, phin, 1.5, r).cpu().numpy()
    assert np.array_equal(zw, zg)
    assert np.isfinite(zw).all() and np.abs(zw).max() > 0


def test_window_apply_refuses_blocks_it_cannot_hold(pfc):
    """FP64 factors and blocks with levels of more than 255 rows run only the global-memory
    apply: asking for the window there fails at creation, and the default falls back."""
    with pytest.raises(pfc.PfcError):
        solver3(pfc, (16, 16, 16), (2, 2, 2), prec=0, apply_variant=1)
    with pytest.raises(pfc.PfcError):
        solver3(pfc, (90, 90, 90), (2, 2, 2), prec=2, apply_variant=1)  # 47^3 blocks: 316-row levels
    assert solver3(pfc, (90, 90, 90), (2, 2, 2), prec=2).tuning()["apply_variant"] == 0
    assert solver3(pfc, (16, 16, 16), (2, 2, 2), prec=0).tuning()["apply_variant"] == 0


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 14, 18), (40, 37, 33)])
def test_float_float_jvp_3d(pfc, shape, prec):
    """The mixed path's 3D JVP (three float-float 7-point passes) against the oracle's FP64
    product: float pairs keep about 2^-44 of the terms, within 1e-11 of the largest entry."""
    Phi = inputs.noise_field(shape, -0.3, 0.4, 31)
    phin = inputs.noise_field(shape, -0.3, 0.4, 32)
    v = inputs.noise_field(shape, 0.0, 1.0, 33)
    s = solver3(pfc, shape, (2, 2, 2), prec=prec)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 2.5, H3, GAMMA3)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 14, 18), (40, 37, 33)])
def test_fp32_jvp_3d(pfc, shape):
    """The opt-in FP32 3D JVP (jvp_fp32 = 1; inputs cut to floats, FP32 passes) against the oracle's
    FP64 product: FP32 rounding of terms up to ih4 |v| in size, bounded at 1e-5 of the largest
    entry (as the 2D FP32 JVP)."""
    Phi = inputs.noise_field(shape, -0.3, 0.4, 31)
    phin = inputs.noise_field(shape, -0.3, 0.4, 32)
    v = inputs.noise_field(shape, 0.0, 1.0, 33)
    s = solver3(pfc, shape, (2, 2, 2), prec=2, jvp_fp32=1)
    Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
    ref = O.jvp(v, Phi, phin, 2.5, H3, GAMMA3)
    np.testing.assert_allclose(Jv, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    assert np.abs(Jv - ref).max() > 1e-12 * np.abs(ref).max()  # it is the FP32 kernel, not the float-float one


def test_steps_3d_fp32_jvp_match_oracle(pfc):
    """Three fixed steps at dt = 0.5 on the 16^3 BCC-seeded field with BF16 factors and the FP32 JVP,
    at the mixed tolerances."""
    shape = (16, 16, 16)
    phi0 = inputs.bcc_seeds_3d(shape, H3, nseeds=1, d0=4 * H3, seed=5)
    s = solver3(pfc, shape, (2, 2, 2), prec=2, jvp_fp32=1)
    s.set_field(phi0)
    infos = [s.step(0.5) for _ in range(3)]
    ref, recs = O.run(phi0, H3, GAMMA3, O.Params(parts=(2, 2, 2), overlap=1, subdomain_solver="ilu0"), 3,
                      fixed_dt=0.5)
    assert np.abs(s.get_field() - ref).max() <= 1e-7
    for inf, rec in zip(infos, recs):
        assert abs(inf["energy"] - rec.energy) <= 1e-9 * abs(rec.energy)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 14, 18)])
def test_neumann_operators_3d(pfc, shape):
    """Mirror walls in 3D (Sec. 2): residual, FP64 and float-float JVP and energy against the
    oracle's operators of the evenly extended fields."""
    Phi = inputs.noise_field(shape, -0.3, 0.4, 41)
    phin = inputs.noise_field(shape, -0.3, 0.4, 42)
    v = inputs.noise_field(shape, 0.0, 1.0, 43)
    s = solver3(pfc, shape, (2, 2, 2), boundary=pfc.PFC_NEUMANN)
    F, nrm = s.residual(Phi, phin, 0.7)
    ref = O.residual(Phi, phin, 0.7, H3, GAMMA3, neumann=True)
    np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    refj = O.jvp(v, Phi, phin, 2.5, H3, GAMMA3, neumann=True)
    np.testing.assert_allclose(s.jvp(Phi, phin, v, 2.5).cpu().numpy(), refj, rtol=0, atol=1e-12 * np.abs(refj).max())
    s2 = solver3(pfc, shape, (2, 2, 2), prec=2, boundary=pfc.PFC_NEUMANN)
    np.testing.assert_allclose(s2.jvp(Phi, phin, v, 2.5).cpu().numpy(), refj, rtol=0, atol=1e-11 * np.abs(refj).max())
    s.set_field(Phi)
    assert s.energy() == pytest.approx(O.energy(Phi, H3, GAMMA3, neumann=True), rel=1e-12)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (2, 0.05)])
@pytest.mark.parametrize("shape,parts", [((16, 16, 16), (2, 2, 2)), ((17, 15, 18), (2, 2, 2)), ((14, 8, 9), (2, 1, 1))])
def test_neumann_precond_3d(pfc, shape, parts, prec, tol):
    """Left-RAS between mirror walls: blocks stop at the walls and A_k is the principal submatrix
    of the Neumann Jacobian (mirror images folded into the block's columns), against the oracle's
    blocks of its assembled Neumann Jacobian."""
    Phi = inputs.noise_field(shape, -0.325, 0.3, 44)
    phin = inputs.noise_field(shape, -0.325, 0.3, 45)
    r = inputs.noise_field(shape, 0.0, 1.0, 46)
    s = solver3(pfc, shape, parts, prec=prec, boundary=pfc.PFC_NEUMANN)
    z = s.precond_apply(Phi, phin, 2.0, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, 2.0, H3, GAMMA3, neumann=True)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1, neumann=True), "left-ras", "ilu0", 0.1).apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol_phi,tol_e", [(0, 1e-8, 1e-10), (2, 1e-7, 1e-9)])
def test_neumann_steps_3d(pfc, prec, tol_phi, tol_e):
    """Three fixed steps at dt = 0.5 between mirror walls on a 16^3 BCC-seeded field."""
    shape = (16, 16, 16)
    phi0 = inputs.bcc_seeds_3d(shape, H3, nseeds=1, d0=4 * H3, seed=5)
    s = solver3(pfc, shape, (2, 2, 2), prec=prec, boundary=pfc.PFC_NEUMANN)
    s.set_field(phi0)
    infos = [s.step(0.5) for _ in range(3)]
    ref, recs = O.run(phi0, H3, GAMMA3, O.Params(parts=(2, 2, 2), overlap=1, subdomain_solver="ilu0", neumann=True),
                      3, fixed_dt=0.5)
    assert np.abs(s.get_field() - ref).max() <= tol_phi
    for inf, rec in zip(infos, recs):
        assert abs(inf["energy"] - rec.energy) <= tol_e * abs(rec.energy)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 14, 18)])
def test_mobility_operators_3d(pfc, shape):
    """Variable mobility M = 1 - phi^2 in 3D (Sec. 3): residual (edge-averaged M of the midpoint)
    and the FP64 JVP with the dM/dPhi term against the oracle, on every path (the mixed path's
    JVP is FP64 too with mobility)."""
    Phi = inputs.noise_field(shape, 0.2, 0.4, 51)
    phin = inputs.noise_field(shape, 0.2, 0.4, 52)
    v = inputs.noise_field(shape, 0.0, 1.0, 53)
    ref = O.residual(Phi, phin, 0.7, H3, GAMMA3, mobility=True)
    refj = O.jvp(v, Phi, phin, 2.5, H3, GAMMA3, mobility=True)
    for prec in (0, 2):
        s = solver3(pfc, shape, (2, 2, 2), prec=prec, mobility=1)
        F, nrm = s.residual(Phi, phin, 0.7)
        np.testing.assert_allclose(F.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert nrm == pytest.approx(np.linalg.norm(ref), rel=1e-12)
        Jv = s.jvp(Phi, phin, v, 2.5).cpu().numpy()
        np.testing.assert_allclose(Jv, refj, rtol=0, atol=1e-12 * np.abs(refj).max())


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (2, 0.05)])
@pytest.mark.parametrize("shape,parts", [((16, 16, 16), (2, 2, 2)), ((17, 16, 15), (2, 2, 2))])
def test_mobility_precond_3d(pfc, shape, parts, prec, tol):
    """Left-RAS with shifted ILU(0) blocks of the mobility Jacobian (the 63-point pattern, entries
    of D_M (L_gamma/2 + Q) and of the dM/dPhi term) against the oracle's blocks of its assembled
    mobility Jacobian."""
    Phi = inputs.noise_field(shape, 0.2, 0.3, 54)
    phin = inputs.noise_field(shape, 0.2, 0.3, 55)
    r = inputs.noise_field(shape, 0.0, 1.0, 56)
    s = solver3(pfc, shape, parts, prec=prec, mobility=1)
    z = s.precond_apply(Phi, phin, 2.0, r).cpu().numpy()
    J = O.assemble_jacobian(Phi, phin, 2.0, H3, GAMMA3, mobility=True)
    ref = O.Schwarz(J, O.decompose(shape, parts, 1), "left-ras", "ilu0", 0.1).apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("prec,tol_phi,tol_e", [(0, 1e-8, 1e-10), (2, 1e-7, 1e-9)])
def test_mobility_steps_3d(pfc, prec, tol_phi, tol_e):
    """Three fixed steps at dt = 0.5 with M = 1 - phi^2 on a 16^3 noisy liquid (|phi| < 1, so M > 0)
    against the oracle (plain FP64 and mixed tolerances)."""
    shape = (16, 16, 16)
    phi0 = inputs.noise_field(shape, -0.325, 0.07, 57)
    s = solver3(pfc, shape, (2, 2, 2), prec=prec, mobility=1)
    s.set_field(phi0)
    infos = [s.step(0.5) for _ in range(3)]
    ref, recs = O.run(phi0, H3, GAMMA3, O.Params(parts=(2, 2, 2), overlap=1, subdomain_solver="ilu0", mobility=True),
                      3, fixed_dt=0.5)
    assert np.abs(s.get_field() - ref).max() <= tol_phi
    for inf, rec in zip(infos, recs):
        assert abs(inf["energy"] - rec.energy) <= tol_e * abs(rec.energy)
