"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form,
a summation identity the scheme is built on, a brute-force dense solve, a
finite-difference derivative, or an order of convergence.  The last test plants
mistakes in the oracle (on the CPU) and checks that a pin catches each one.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pfc_oracle as O
from paper_1703_01202_gb300 import inputs

H2 = math.pi / 4
GAMMA = 0.25


def rand_field(shape, seed, mean=0.1, amp=0.3):
    return inputs.noise_field(shape, mean, amp, seed)


def kappa(ks, ns, h):
    """Symbol of -Delta_d on the Fourier mode with integer wave numbers ks."""
    return sum(4.0 / h**2 * math.sin(math.pi * k / n) ** 2 for k, n in zip(ks, ns))


def mode(shape, ks, h):
    """cos(sum_a 2 pi k_a x_a / L_a) on the cell centres."""
    coords = inputs.cell_centres(shape, h)
    arg = 0.0
    for c, k, n in zip(coords, ks, shape):
        arg = arg + 2.0 * math.pi * k * c / (n * h)
    return np.cos(arg)


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("shape,ks", [((12, 16), (2, 3)), ((6, 10, 8), (1, 4, 3))])
def test_laplacian_fourier_symbol(shape, ks):
    """Delta_d cos(k.x) = -kappa cos(k.x), kappa = sum 4/h^2 sin^2(pi k/N) (Sec. 3)."""
    h = 0.7
    u = mode(shape, ks, h)
    lam = kappa(ks, shape, h)
    np.testing.assert_allclose(O.lap(u, h), -lam * u, rtol=0, atol=1e-12 * lam)
    # L_gamma acts as (1-g) - 2 kappa + kappa^2 (Eq. discretedG)
    s = (1 - GAMMA) - 2 * lam + lam**2
    np.testing.assert_allclose(O.L_gamma(u, h, GAMMA), s * u, rtol=0, atol=1e-11 * (1 + lam**2))


def test_energy_closed_forms():
    """F_d of a constant and of one Fourier mode (Eqs. relations, freeenergy)."""
    shape = (16, 24)
    h = 0.6
    area = h * h * shape[0] * shape[1]
    c = 0.37
    assert O.energy(np.full(shape, c), h, GAMMA) == pytest.approx(
        area * ((1 - GAMMA) * c * c / 2 + c**4 / 4), rel=1e-13)
    # phi = A cos(2 pi k x / L) with 2k, 4k not multiples of N: mean of cos^2 = 1/2, cos^4 = 3/8
    A = 0.3
    ks = (0, 5)
    phi = A * mode(shape, ks, h)
    lam = kappa(ks, shape, h)
    expect = area * (A * A / 4 * ((1 - GAMMA) - 2 * lam + lam * lam) + 3 * A**4 / 32)
    assert O.energy(phi, h, GAMMA) == pytest.approx(expect, rel=1e-12)
    assert O.mass(phi + 0.2, h) == pytest.approx(0.2 * area, rel=1e-12)


@pytest.mark.parametrize("shape", [(10, 12), (6, 8, 7)])
def test_dvd_identity(shape):
    """Eq. (DVD): h^d sum [G_d(phi1) - G_d(phi0)] = h^d sum mu(phi1, phi0)(phi1 - phi0)."""
    h = 0.8
    p1 = rand_field(shape, 1)
    p0 = rand_field(shape, 2)
    lhs = O.energy(p1, h, GAMMA) - O.energy(p0, h, GAMMA)
    rhs = float(np.sum(O.mu_dvd(p1, p0, h, GAMMA) * (p1 - p0))) * h ** len(shape)
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12 * abs(O.energy(p0, h, GAMMA)))


@pytest.mark.parametrize("shape", [(10, 12), (6, 8, 7)])
def test_summation_by_parts(shape):
    """Eq. (summation) with M = 1: sum g Delta_d g = -sum_axes sum (D^+ g)^2."""
    h = 0.9
    g = rand_field(shape, 3)
    lhs = float(np.sum(g * O.lap(g, h)))
    rhs = -sum(float(np.sum(O.d_plus(g, ax, h) ** 2)) for ax in range(len(shape)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ---------------------------------------------------------------- Jacobian
def test_jacobian_matches_finite_differences():
    """Analytic J v against central differences of F (Eq. Jacobi)."""
    shape = (12, 10)
    Phi = rand_field(shape, 4, 0.2, 0.4)
    phin = rand_field(shape, 5, 0.2, 0.4)
    v = rand_field(shape, 6, 0.0, 1.0)
    dt = 0.7
    Jv = O.jvp(v, Phi, phin, dt, H2, GAMMA)
    eps = 1e-5 * np.linalg.norm(Phi) / np.linalg.norm(v)
    fd = (O.residual(Phi + eps * v, phin, dt, H2, GAMMA) - O.residual(Phi - eps * v, phin, dt, H2, GAMMA)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) <= 1e-8 * np.linalg.norm(Jv)
    J = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA)
    np.testing.assert_allclose((J @ v.ravel()).reshape(shape), Jv, rtol=0, atol=1e-13 * np.abs(Jv).max())
    # 3D as well
    s3 = (6, 7, 8)
    Phi3, phin3, v3 = rand_field(s3, 7), rand_field(s3, 8), rand_field(s3, 9, 0.0, 1.0)
    Jv3 = O.jvp(v3, Phi3, phin3, dt, H2, GAMMA)
    fd3 = (O.residual(Phi3 + eps * v3, phin3, dt, H2, GAMMA) - O.residual(Phi3 - eps * v3, phin3, dt, H2, GAMMA)) / (2 * eps)
    assert np.linalg.norm(Jv3 - fd3) <= 1e-8 * np.linalg.norm(Jv3)


# ---------------------------------------------------------------- Schwarz pieces
@pytest.mark.parametrize("shape,parts,overlap", [((16, 20), (2, 3), 1), ((17, 16), (3, 2), 2), ((10, 10, 10), (2, 2, 2), 1)])
def test_improved_bc_equals_principal_submatrix(shape, parts, overlap):
    """The subdomain problem with phi = 0 on the 3-layer ring (Sec. 4, improved
    boundary condition) gives exactly A_k = R J R^T (Eq. Ak) whenever the block
    plus its ring does not wrap onto itself (block width + 3 <= grid width)."""
    Phi, phin = rand_field(shape, 10), rand_field(shape, 11)
    dt = 2.0
    J = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA)
    blocks = O.decompose(shape, parts, overlap)
    for blk in blocks[:3]:
        A1 = O.subdomain_matrix(J, blk)
        A2 = O.subdomain_matrix_improved_bc(Phi, phin, dt, H2, GAMMA, blk)
        np.testing.assert_allclose(A2, A1, rtol=0, atol=1e-13 * np.abs(A1).max())


def test_decomposition_covers_grid_once():
    """Cores partition the grid (uneven splits give the extra cell to the first cores)."""
    for shape, parts in [((64, 64), (4, 4)), ((37, 50), (3, 7)), ((10, 11, 9), (2, 3, 2))]:
        blocks = O.decompose(shape, parts, 1)
        hits = np.zeros(int(np.prod(shape)), dtype=int)
        for b in blocks:
            hits[b.core_idx] += 1
        assert np.all(hits == 1)
    assert O.split_axis(256, 7) == [(0, 37), (37, 37), (74, 37), (111, 37), (148, 36), (184, 36), (220, 36)]


def test_single_block_ras_is_exact_inverse():
    """One subdomain covering the periodic grid: H^{-1} = J^{-1}, so GMRES needs one iteration."""
    shape = (10, 12)
    Phi, phin = rand_field(shape, 12), rand_field(shape, 13)
    J = O.assemble_jacobian(Phi, phin, 1.0, H2, GAMMA)
    pre = O.Schwarz(J, O.decompose(shape, (1, 1), 0), "left-ras", "lu")
    b = rand_field(shape, 14, 0.0, 1.0)
    res = O.gmres_right(lambda v: (J @ v.ravel()).reshape(shape), pre.apply, b, 1e-12 * np.linalg.norm(b))
    assert res.iterations == 1
    np.testing.assert_allclose(res.x.ravel(), np.linalg.solve(J.toarray(), b.ravel()), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("neumann", [False, True])
def test_ras_variants_match_definitions(neumann):
    """AS / left-RAS / right-RAS (Eqs. invM, ras, ash) against explicit sums of
    restriction matrices times dense block inverses; periodic, and between Neumann walls
    (wall-clipped blocks of the Neumann Jacobian)."""
    shape = (12, 12)
    Phi, phin = rand_field(shape, 15), rand_field(shape, 16)
    J = O.assemble_jacobian(Phi, phin, 0.5, H2, GAMMA, neumann=neumann)
    blocks = O.decompose(shape, (2, 3), 1, neumann=neumann)
    n = Phi.size
    r = rand_field(shape, 17, 0.0, 1.0).ravel()
    for kind in ("as", "left-ras", "right-ras"):
        M = np.zeros((n, n))
        for blk in blocks:
            Rd = np.zeros((blk.block_idx.size, n))
            Rd[np.arange(blk.block_idx.size), blk.block_idx] = 1.0
            R0 = Rd * blk.core_mask[:, None]
            Ainv = np.linalg.inv(J.toarray()[np.ix_(blk.block_idx, blk.block_idx)])
            left = R0 if kind == "left-ras" else Rd
            right = R0 if kind == "right-ras" else Rd
            M += left.T @ Ainv @ right
        z = O.Schwarz(J, blocks, kind, "lu").apply(r.reshape(shape)).ravel()
        np.testing.assert_allclose(z, M @ r, rtol=1e-10, atol=1e-12 * np.abs(M @ r).max())


def test_ilu0_on_banded_pattern_is_exact_lu():
    """ILU(0) equals exact LU when the pattern already holds all fill (a
    tridiagonal matrix); and its factors reproduce A on the pattern."""
    n = 30
    rng = np.random.default_rng(0)
    A = sp.diags([rng.uniform(-1, 1, n - 1), 4 + rng.uniform(0, 1, n), rng.uniform(-1, 1, n - 1)], [-1, 0, 1], format="csr")
    LU = O.ilu0(A)
    b = rng.uniform(-1, 1, n)
    np.testing.assert_allclose(O.ilu0_solve(LU, b), np.linalg.solve(A.toarray(), b), rtol=1e-12)
    # 2D 5-point matrix: (L U)_ij = a_ij on the pattern
    m = 6
    T = sp.diags([-np.ones(m - 1), 4 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    A2 = (sp.kron(sp.identity(m), T) + sp.kron(sp.diags([-np.ones(m - 1), -np.ones(m - 1)], [-1, 1]), sp.identity(m))).tocsr()
    LU2 = O.ilu0(A2).toarray()
    L = np.tril(LU2, -1) + np.eye(m * m)
    U = np.triu(LU2)
    prod = L @ U
    mask = A2.toarray() != 0
    np.testing.assert_allclose(prod[mask], A2.toarray()[mask], atol=1e-13)


def test_shifted_ilu0_is_ilu0_of_the_shifted_block():
    """The 3D reading: 'ilu0' with ilu_shift s factors A_k + s mean|diag A_k| I.  The
    shift changes the apply, and the apply equals unshifted ILU(0) of the block
    matrix with the shift added to its diagonal by hand."""
    shape = (10, 10, 10)
    Phi, phin = rand_field(shape, 30), rand_field(shape, 31)
    J = O.assemble_jacobian(Phi, phin, 0.5, 80 * math.pi / 256, 0.3)
    blocks = O.decompose(shape, (2, 2, 2), 1)
    r = rand_field(shape, 32, 0.0, 1.0)
    z0 = O.Schwarz(J, blocks, "left-ras", "ilu0", 0.0).apply(r)
    z1 = O.Schwarz(J, blocks, "left-ras", "ilu0", 0.2).apply(r)
    assert np.linalg.norm(z1 - z0) > 1e-3 * np.linalg.norm(z0)  # the shift changes the factors
    # same block, shift folded into the matrix by hand, unshifted ILU(0): identical apply
    blk = blocks[0]
    A = O.subdomain_matrix(J, blk)
    As = A + 0.2 * np.mean(np.abs(np.diag(A))) * np.eye(A.shape[0])
    rows, cols = np.nonzero(O.block_pattern(blk))
    LU = O.ilu0(sp.csr_matrix((As[rows, cols], (rows, cols)), shape=As.shape))
    sol = O.ilu0_solve(LU, r.ravel()[blk.block_idx])
    np.testing.assert_allclose(z1.ravel()[blk.core_idx], sol[blk.core_mask], rtol=1e-13, atol=1e-15)


def test_ilu0_schwarz_between_walls_is_per_block_ilu0():
    """Between mirror walls the blocks stop at the walls (blocks of several extents): the
    Schwarz 'ilu0' apply, which factors the blocks of one extent side by side, equals ILU(0) of
    each block's own shifted matrix solved on its own, block by block (left-RAS: core rows)."""
    shape = (12, 11, 10)
    Phi, phin = rand_field(shape, 33), rand_field(shape, 34)
    J = O.assemble_jacobian(Phi, phin, 0.5, 80 * math.pi / 256, 0.3, neumann=True)
    blocks = O.decompose(shape, (2, 2, 2), 1, neumann=True)
    assert len({b.dims for b in blocks}) > 1 and all(b.dims[0] == 7 for b in blocks)  # 6 + 1 at each wall
    r = rand_field(shape, 35, 0.0, 1.0)
    z = O.Schwarz(J, blocks, "left-ras", "ilu0", 0.1).apply(r)
    ref = np.zeros(r.size)
    for blk in blocks:
        A = O.subdomain_matrix(J, blk)
        As = A + 0.1 * np.mean(np.abs(np.diag(A))) * np.eye(A.shape[0])
        rows, cols = np.nonzero(O.block_pattern(blk))
        assert not np.any(As[~O.block_pattern(blk)])  # the folded wall rows stay in the radius-3 pattern
        LU = O.ilu0(sp.csr_matrix((As[rows, cols], (rows, cols)), shape=As.shape))
        ref[blk.core_idx] = O.ilu0_solve(LU, r.ravel()[blk.block_idx])[blk.core_mask]
    np.testing.assert_allclose(z.ravel(), ref, rtol=1e-13, atol=1e-15)


def test_gmres_unpreconditioned_matches_dense_solve():
    """GMRES with H = I to 1e-14 against a dense solve (restart exercised)."""
    shape = (8, 8)
    Phi, phin = rand_field(shape, 18), rand_field(shape, 19)
    J = O.assemble_jacobian(Phi, phin, 0.3, H2, GAMMA)
    b = rand_field(shape, 20, 0.0, 1.0)
    res = O.gmres_right(lambda v: (J @ v.ravel()).reshape(shape), lambda v: v, b, 1e-14 * np.linalg.norm(b), restart=10)
    assert res.converged
    np.testing.assert_allclose(res.x.ravel(), np.linalg.solve(J.toarray(), b.ravel()), rtol=0, atol=1e-11 * np.abs(b).max())


# ---------------------------------------------------------------- full step
def dense_newton(phin, dt, h, gamma, tol=1e-14):
    """Brute force: Newton with the dense Jacobian solved by LAPACK."""
    Phi = phin.copy()
    for _ in range(50):
        F = O.residual(Phi, phin, dt, h, gamma)
        if np.linalg.norm(F) <= tol:
            break
        J = O.assemble_jacobian(Phi, phin, dt, h, gamma).toarray()
        Phi = Phi - np.linalg.solve(J, F.ravel()).reshape(Phi.shape)
    return Phi


@pytest.mark.parametrize("shape,parts,solver,h,dt", [((8, 8), (2, 2), "lu", H2, 0.5),
                                                     ((10, 10, 10), (2, 2, 2), "ilu0", 80 * math.pi / 256, 0.1)])
def test_nks_matches_dense_direct_solve(shape, parts, solver, h, dt):
    """NKS step (Newton + right-preconditioned GMRES + left-RAS) against Newton
    with dense direct solves, to 1e-12 (tight tolerances on both sides).  3D uses
    ILU(0) subdomain solves at the 3D test's spacing and a dt where ILU(0) of the
    radius-3 block matrix has positive pivots."""
    phin = inputs.noise_field(shape, 0.07, 0.07, 21)
    p = O.Params(newton_rtol=1e-13, gmres_rtol=1e-8, parts=parts, overlap=1, subdomain_solver=solver)
    Phi, info = O.newton_solve(phin, dt, h, GAMMA, p)
    ref = dense_newton(phin, dt, h, GAMMA)
    assert info.converged and info.newton_its >= 2
    assert np.abs(Phi - ref).max() <= 1e-12


@pytest.mark.parametrize("dt", [1e-3, 1e-2, 0.1, 1.0, 5.0, 100.0])
def test_energy_law_and_decrease(dt):
    """Proposition: F_d(phi^{n+1}) <= F_d(phi^n) for every dt, and the exact
    balance F1 - F0 = -dt h^2 sum_axes sum (D^+ mu)^2 + dt h^2 sum mu F(phi1).
    (dt near 2/|kappa S| for a grid mode makes J singular for this liquid at
    gamma = 0.25; such dt, e.g. 10 here, are left out.)"""
    shape = (16, 16)
    phin = inputs.noise_field(shape, 0.07, 0.07, 22)
    p = O.Params(parts=(2, 2), overlap=1, newton_rtol=1e-12)
    phi1, info = O.newton_solve(phin, dt, H2, GAMMA, p)
    assert info.converged
    F0, F1 = O.energy(phin, H2, GAMMA), O.energy(phi1, H2, GAMMA)
    mu = O.mu_dvd(phi1, phin, H2, GAMMA)
    diss = sum(float(np.sum(O.d_plus(mu, ax, H2) ** 2)) for ax in range(2))
    rest = float(np.sum(mu * O.residual(phi1, phin, dt, H2, GAMMA)))
    assert F1 - F0 == pytest.approx(-dt * H2**2 * diss + dt * H2**2 * rest, rel=1e-9, abs=1e-12 * abs(F0))
    assert F1 <= F0


def test_mass_conservation():
    """Sum phi is conserved (Sec. 3): with the zero-mean update to 1e-12; and,
    for a loosely solved step without it, the drift equals dt h^2 sum F(phi^{n+1})
    (sum Delta_d = 0 on the periodic grid)."""
    shape = (16, 16)
    phi0 = inputs.noise_field(shape, 0.07, 0.07, 23)
    p = O.Params(parts=(2, 2), overlap=1)
    phi, recs = O.run(phi0, H2, GAMMA, p, 8, fixed_dt=0.5)
    m0 = O.mass(phi0, H2)
    assert all(abs(r.mass - m0) <= 1e-12 * max(1.0, abs(m0)) for r in recs)
    p2 = O.Params(parts=(2, 2), overlap=1, mass_projection=False, newton_rtol=1e-2, gmres_rtol=0.3)
    phi1, _ = O.newton_solve(phi0, 0.5, H2, GAMMA, p2)
    drift = O.mass(phi1, H2) - m0
    expect = 0.5 * H2**2 * float(np.sum(O.residual(phi1, phi0, 0.5, H2, GAMMA)))
    assert abs(drift - expect) <= 1e-13 * max(1.0, abs(m0))


def test_constant_is_fixed_point():
    """A constant field is a steady state: F = 0, zero Newton iterations."""
    phin = np.full((12, 12), 0.3)
    assert np.abs(O.residual(phin, phin, 1.0, H2, GAMMA)).max() < 1e-14
    phi1, info = O.newton_solve(phin, 1.0, H2, GAMMA, O.Params(parts=(2, 2)))
    assert info.newton_its == 0 and np.array_equal(phi1, phin)


@pytest.mark.parametrize("dt", [0.05, 1.0, 20.0])
def test_fourier_mode_crank_nicolson_multiplier(dt):
    """Small-amplitude mode: the scheme is Crank-Nicolson on the linearised
    equation, so phi1 = g phi0 with g = (1 - dt kappa S/2)/(1 + dt kappa S/2),
    S = (1-gamma) - 2 kappa + kappa^2 (Eqs. discretedG, NSOP)."""
    shape = (16, 16)
    h = 1.1
    ks = (1, 2)
    phi0 = 1e-6 * mode(shape, ks, h)
    lam = kappa(ks, shape, h)
    S = (1 - GAMMA) - 2 * lam + lam * lam
    g = (1 - 0.5 * dt * lam * S) / (1 + 0.5 * dt * lam * S)
    p = O.Params(parts=(2, 2), newton_rtol=1e-13, gmres_rtol=1e-12)
    phi1, info = O.newton_solve(phi0, dt, h, GAMMA, p)
    np.testing.assert_allclose(phi1, g * phi0, rtol=0, atol=1e-9 * 1e-6)


def test_adaptive_dt_formula():
    """Eq. (sencondt) with hand-computed values."""
    p = O.Params(dt_min=0.01, dt_max=10.0, eta=5000.0)
    # F' = (E_n - E_nm1)/dt_prev = -0.02/0.5 = -0.04 ; 1 + 5000*0.0016 = 9 -> 10/3
    assert O.adaptive_dt(-1.02, -1.0, 0.5, p) == pytest.approx(10.0 / 3.0, rel=1e-15)
    assert O.adaptive_dt(-1.0, -1.0, 0.5, p) == 10.0
    assert O.adaptive_dt(-100.0, 0.0, 0.01, p) == 0.01


# ---------------------------------------------------------------- orders of accuracy
def test_second_order_in_space():
    """Sec. 5 accuracy test (sine initial value on [0,32]^2, gamma = 0.025) with
    ratio-3 refinement so that cell centres coincide (coarse cell i sits on fine
    cell 3i+1, or 9i+4 two levels down): the error ratio between successive
    grids approaches 9 (second order).  Smaller grids and final time than the
    paper's 1024^2 reference, same initial value."""
    gamma = 0.025
    L = 32.0
    dt, steps = 0.1, 3
    sols = {}
    for n, parts, ov in [(12, (1, 1), 0), (36, (1, 1), 0), (108, (2, 2), 2)]:
        h = L / n
        phi0 = inputs.sine_field((n, n), h)
        p = O.Params(parts=parts, overlap=ov, newton_rtol=1e-10, newton_atol=1e-8, gmres_rtol=1e-8)
        sols[n], _ = O.run(phi0, h, gamma, p, steps, fixed_dt=dt)
    ref = sols[108]
    e12 = np.linalg.norm(sols[12] - ref[4::9, 4::9]) / np.linalg.norm(ref[4::9, 4::9])
    e36 = np.linalg.norm(sols[36] - ref[1::3, 1::3]) / np.linalg.norm(ref[1::3, 1::3])
    # C h^2 (1 - 1/81) against C (h/3)^2 (1 - 1/9): ratio -> 10 asymptotically
    assert 8.5 < e12 / e36 < 11.0


def test_second_order_in_time():
    """Temporal accuracy (Sec. 5): errors against a dt/64 reference fall by ~4 per halving."""
    gamma = 0.025
    n = 32
    h = 1.0
    phi0 = inputs.sine_field((n, n), h)
    T = 1.0
    p = O.Params(parts=(2, 2), overlap=1, newton_rtol=1e-12, gmres_rtol=1e-8)
    ref, _ = O.run(phi0, h, gamma, p, 128, fixed_dt=T / 128)
    errs = []
    for m in (4, 8, 16):
        sol, _ = O.run(phi0, h, gamma, p, m, fixed_dt=T / m)
        errs.append(np.linalg.norm(sol - ref) / np.linalg.norm(ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped term, a wrong sign or a wrong factor in the oracle trips a pin."""
    shape = (10, 12)
    h = 0.8
    p1, p0 = rand_field(shape, 1), rand_field(shape, 2)

    def dvd_gap():
        lhs = O.energy(p1, h, GAMMA) - O.energy(p0, h, GAMMA)
        rhs = float(np.sum(O.mu_dvd(p1, p0, h, GAMMA) * (p1 - p0))) * h * h
        return abs(lhs - rhs) / abs(lhs)

    assert dvd_gap() < 1e-12
    orig_mu = O.mu_dvd
    # dropped phi^n^3 term
    monkeypatch.setattr(O, "mu_dvd", lambda P, q, hh, g: orig_mu(P, q, hh, g) - q**3 / 4)
    assert dvd_gap() > 1e-6
    monkeypatch.setattr(O, "mu_dvd", orig_mu)
    # wrong sign of the 2 Delta term in L_gamma
    orig_lg = O.L_gamma
    monkeypatch.setattr(O, "L_gamma", lambda u, hh, g: orig_lg(u, hh, g) - 4.0 * O.lap(u, hh))
    assert dvd_gap() > 1e-6
    monkeypatch.setattr(O, "L_gamma", orig_lg)
    # gradient term of G_d halved
    orig_le = O.local_energy

    def bad_le(phi, hh, g):
        out = orig_le(phi, hh, g)
        for ax in range(phi.ndim):
            out += 0.25 * (O.d_plus(phi, ax, hh) ** 2 + O.d_minus(phi, ax, hh) ** 2)
        return out

    monkeypatch.setattr(O, "local_energy", bad_le)
    assert dvd_gap() > 1e-6
    monkeypatch.setattr(O, "local_energy", orig_le)
    # transposed / wrong q in the Jacobian: finite-difference pin fails
    Phi, phin, v = rand_field(shape, 4, 0.2, 0.4), rand_field(shape, 5, 0.2, 0.4), rand_field(shape, 6, 0.0, 1.0)
    orig_q = O.jac_coeff
    monkeypatch.setattr(O, "jac_coeff", lambda P, q: (3 * q**2 + 2 * P * q + P**2) / 4)
    Jv = O.jvp(v, Phi, phin, 0.7, h, GAMMA)
    eps = 1e-5
    fd = (O.residual(Phi + eps * v, phin, 0.7, h, GAMMA) - O.residual(Phi - eps * v, phin, 0.7, h, GAMMA)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) > 1e-4 * np.linalg.norm(Jv)
    monkeypatch.setattr(O, "jac_coeff", orig_q)


def test_safeguarded_extrapolation_reaches_the_plain_solution():
    """With the extrapolated (safeguarded) guess the Newton tolerance stays the
    plain method's, eps_r ||F(phi^n)||: both runs reach the same discrete
    solution within that tolerance, and the guess never costs iterations here."""
    h, gamma = math.pi / 4, 0.25
    phi0 = inputs.noise_field((24, 24), 0.07, 0.07, 31)
    p = O.Params(parts=(2, 2), overlap=1)
    a, ra = O.run(phi0, h, gamma, p, 4, fixed_dt=0.5, guess="prev")
    b, rb = O.run(phi0, h, gamma, p, 4, fixed_dt=0.5, guess="extrap")
    assert np.abs(a - b).max() <= 1e-9
    assert sum(r.newton_its for r in rb) <= sum(r.newton_its for r in ra)


# ---------------------------------------------------------------- variable mobility M = 1 - phi^2
def test_mobility_operator_is_conservative_symmetric_and_sums_by_parts():
    """(div M grad)_d of Sec. 3 with edge-averaged M: sums to zero (mass), is symmetric, and
    sum u (div M grad)_d u = -sum over edges M_edge (D^+ u)^2 (summation by parts, the
    dissipation in the energy law); with M constant it is M Delta_d."""
    shape = (12, 10)
    u, v = rand_field(shape, 21, 0.0, 1.0), rand_field(shape, 22, 0.0, 1.0)
    Mn = 0.5 + 0.4 * rand_field(shape, 23, 0.0, 1.0)
    Du, Dv = O.div_m_grad(u, Mn, H2), O.div_m_grad(v, Mn, H2)
    assert abs(float(np.sum(Du))) <= 1e-12 * float(np.abs(Du).sum())
    assert float(np.sum(v * Du)) == pytest.approx(float(np.sum(u * Dv)), rel=1e-12)
    edges = 0.0
    for ax in range(2):
        me = 0.5 * (Mn + np.roll(Mn, -1, axis=ax))
        edges += float(np.sum(me * O.d_plus(u, ax, H2) ** 2))
    assert float(np.sum(u * Du)) == pytest.approx(-edges, rel=1e-12)
    np.testing.assert_allclose(O.div_m_grad(u, np.full(shape, 0.91), H2), 0.91 * O.lap(u, H2), rtol=0,
                               atol=1e-13 * np.abs(O.lap(u, H2)).max())


def test_mobility_jacobian_matches_finite_differences():
    """With M = 1 - phi^2 at (Phi + phi^n)/2 the Jacobian gains the dM/dPhi term; the analytic
    J v against central differences of F, and the assembled matrix against J v."""
    shape = (12, 10)
    Phi = rand_field(shape, 24, 0.2, 0.4)
    phin = rand_field(shape, 25, 0.2, 0.4)
    v = rand_field(shape, 26, 0.0, 1.0)
    dt = 0.7
    Jv = O.jvp(v, Phi, phin, dt, H2, GAMMA, mobility=True)
    eps = 1e-5 * np.linalg.norm(Phi) / np.linalg.norm(v)
    fd = (O.residual(Phi + eps * v, phin, dt, H2, GAMMA, mobility=True)
          - O.residual(Phi - eps * v, phin, dt, H2, GAMMA, mobility=True)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) <= 1e-8 * np.linalg.norm(Jv)
    J = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA, mobility=True)
    np.testing.assert_allclose((J @ v.ravel()).reshape(shape), Jv, rtol=0, atol=1e-12 * np.abs(Jv).max())
    # and it differs from the constant-mobility Jacobian (the term is not dropped)
    assert np.linalg.norm(Jv - O.jvp(v, Phi, phin, dt, H2, GAMMA)) > 1e-3 * np.linalg.norm(Jv)


@pytest.mark.parametrize("dt", [0.05, 1.0])
def test_mobility_fourier_mode_multiplier(dt):
    """Small mode on a uniform field phi_bar = 0.3: linearised, the scheme is Crank-Nicolson with
    mobility M(phi_bar) = 1 - phi_bar^2 and the cubic term's slope 3 phi_bar^2 added to S:
    phi1 - phi_bar = g (phi0 - phi_bar), g = (1 - dt M kappa S/2)/(1 + dt M kappa S/2)."""
    shape = (16, 16)
    h = 1.1
    ks = (1, 2)
    pbar = 0.3
    d0 = 1e-6 * mode(shape, ks, h)
    lam = kappa(ks, shape, h)
    S = (1 - GAMMA) + 3 * pbar ** 2 - 2 * lam + lam * lam
    M = 1 - pbar ** 2
    g = (1 - 0.5 * dt * M * lam * S) / (1 + 0.5 * dt * M * lam * S)
    p = O.Params(parts=(2, 2), newton_rtol=1e-13, gmres_rtol=1e-12, mobility=True)
    phi1, info = O.newton_solve(pbar + d0, dt, h, GAMMA, p)
    np.testing.assert_allclose(phi1 - pbar, g * d0, rtol=0, atol=1e-5 * 1e-6)
    # the constant-mobility solve of the same step misses M (a plausible dropped term)
    assert abs(g - (1 - 0.5 * dt * lam * S) / (1 + 0.5 * dt * lam * S)) > 1e-4


def test_mobility_steps_conserve_mass_and_decrease_energy():
    """Two Newton steps with M = 1 - phi^2 on a noisy field: mass to 1e-12 and a non-increasing
    discrete energy (Sec. 3 energy law; the dissipation is sum M_edge (D^+ mu)^2 >= 0 while M > 0)."""
    shape = (16, 16)
    phi = 0.07 + 0.07 * rand_field(shape, 27, 0.0, 1.0)
    p = O.Params(parts=(2, 2), mobility=True)
    e0, m0 = O.energy(phi, H2, GAMMA), O.mass(phi, H2)
    for _ in range(2):
        phi, info = O.newton_solve(phi, 0.5, H2, GAMMA, p)
        assert info.converged
        e1 = O.energy(phi, H2, GAMMA)
        assert e1 <= e0 + 1e-13 * abs(e0)
        assert abs(O.mass(phi, H2) - m0) <= 1e-12 * max(1.0, abs(m0))
        e0 = e1


# ---------------------------------------------------------------- variable mobility in 3D
def test_mobility_3d_on_a_field_constant_along_one_axis_is_the_2d_operator():
    """A 3D field constant along one axis has no flux across that axis: the 3D residual and JVP
    with M = 1 - phi^2 equal the 2D ones of the remaining two axes, for each choice of the constant
    axis (so every axis of the 3D operator is exercised against the pinned 2D one)."""
    rng_shape2 = (10, 12)
    Phi2 = rand_field(rng_shape2, 61, 0.2, 0.4)
    phin2 = rand_field(rng_shape2, 62, 0.2, 0.4)
    v2 = rand_field(rng_shape2, 63, 0.0, 1.0)
    dt = 0.6
    F2 = O.residual(Phi2, phin2, dt, H2, GAMMA, mobility=True)
    J2 = O.jvp(v2, Phi2, phin2, dt, H2, GAMMA, mobility=True)
    for ax in range(3):
        rep = lambda a: np.repeat(np.expand_dims(a, ax), 5, axis=ax)  # noqa: E731
        F3 = O.residual(rep(Phi2), rep(phin2), dt, H2, GAMMA, mobility=True)
        J3 = O.jvp(rep(v2), rep(Phi2), rep(phin2), dt, H2, GAMMA, mobility=True)
        np.testing.assert_allclose(F3, rep(F2), rtol=0, atol=1e-12 * np.abs(F2).max())
        np.testing.assert_allclose(J3, rep(J2), rtol=0, atol=1e-12 * np.abs(J2).max())


def test_mobility_3d_jacobian_matches_finite_differences():
    """3D, M = 1 - phi^2: the analytic J v against central differences of F, the assembled
    matrix against J v, and the dM/dPhi term present."""
    shape = (6, 7, 8)
    Phi = rand_field(shape, 64, 0.2, 0.4)
    phin = rand_field(shape, 65, 0.2, 0.4)
    v = rand_field(shape, 66, 0.0, 1.0)
    dt = 0.7
    Jv = O.jvp(v, Phi, phin, dt, H2, GAMMA, mobility=True)
    eps = 1e-5 * np.linalg.norm(Phi) / np.linalg.norm(v)
    fd = (O.residual(Phi + eps * v, phin, dt, H2, GAMMA, mobility=True)
          - O.residual(Phi - eps * v, phin, dt, H2, GAMMA, mobility=True)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) <= 1e-8 * np.linalg.norm(Jv)
    J = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA, mobility=True)
    np.testing.assert_allclose((J @ v.ravel()).reshape(shape), Jv, rtol=0, atol=1e-12 * np.abs(Jv).max())
    assert np.linalg.norm(Jv - O.jvp(v, Phi, phin, dt, H2, GAMMA)) > 1e-3 * np.linalg.norm(Jv)
    # the block matrices keep the 63-point pattern of the constant-mobility Jacobian
    J1 = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA)
    assert set(zip(*J.nonzero())) <= set(zip(*J1.nonzero()))


@pytest.mark.parametrize("dt", [0.05, 1.0])
def test_mobility_3d_fourier_mode_multiplier(dt):
    """3D small mode on phi_bar = 0.3 with M = 1 - phi^2: Crank-Nicolson with M(phi_bar) and the cubic
    slope 3 phi_bar^2, g = (1 - dt M kappa S/2)/(1 + dt M kappa S/2), solved with the shifted-ILU(0)
    Schwarz blocks of the 3D path."""
    shape = (16, 16, 16)
    h = 1.1
    ks = (1, 2, 1)
    pbar = 0.3
    d0 = 1e-6 * mode(shape, ks, h)
    lam = kappa(ks, shape, h)
    S = (1 - GAMMA) + 3 * pbar ** 2 - 2 * lam + lam * lam
    M = 1 - pbar ** 2
    g = (1 - 0.5 * dt * M * lam * S) / (1 + 0.5 * dt * M * lam * S)
    p = O.Params(parts=(2, 2, 2), newton_rtol=1e-13, gmres_rtol=1e-12, mobility=True, subdomain_solver="ilu0")
    phi1, info = O.newton_solve(pbar + d0, dt, h, GAMMA, p)
    np.testing.assert_allclose(phi1 - pbar, g * d0, rtol=0, atol=1e-5 * 1e-6)
    # a solve that dropped M would give the constant-mobility multiplier
    assert abs(g - (1 - 0.5 * dt * lam * S) / (1 + 0.5 * dt * lam * S)) > 1e-4


def test_mobility_3d_steps_conserve_mass_and_decrease_energy():
    """Two 3D Newton steps with M = 1 - phi^2 and shifted-ILU(0) blocks: mass to 1e-12 and a
    non-increasing discrete energy."""
    shape = (16, 16, 16)
    h = 80 * math.pi / 256
    phi = -0.325 + 0.07 * rand_field(shape, 67, 0.0, 1.0)
    p = O.Params(parts=(2, 2, 2), mobility=True, subdomain_solver="ilu0")
    e0, m0 = O.energy(phi, h, 0.3), O.mass(phi, h)
    for _ in range(2):
        phi, info = O.newton_solve(phi, 0.5, h, 0.3, p)
        assert info.converged
        e1 = O.energy(phi, h, 0.3)
        assert e1 <= e0 + 1e-13 * abs(e0)
        assert abs(O.mass(phi, h) - m0) <= 1e-12 * max(1.0, abs(m0))
        e0 = e1


# ---------------------------------------------------------------- Neumann-type walls (Sec. 2)
def neumann_lap_matrix(shape, h):
    """Textbook cell-centred Neumann Laplacian, built by hand: per axis the tridiagonal
    (1, -2, 1)/h^2 with the ghost folded into the end rows (-1 instead of -2), then the
    Kronecker sum over the axes.  Independent of the oracle's even-extension route."""
    mats = []
    for n in shape:
        T = np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        T[0, 0] = T[-1, -1] = -1.0
        mats.append(T / (h * h))
    out = np.zeros((int(np.prod(shape)),) * 2)
    for ax, T in enumerate(mats):
        left = np.eye(int(np.prod(shape[:ax])))
        right = np.eye(int(np.prod(shape[ax + 1:])))
        out += np.kron(np.kron(left, T), right)
    return out


def neumann_parts(shape, h):
    Lap = neumann_lap_matrix(shape, h)
    Lg = (1 - GAMMA) * np.eye(Lap.shape[0]) + 2 * Lap + Lap @ Lap
    return Lap, Lg


def neumann_residual_by_hand(Phi, phin, dt, h):
    Lap, Lg = neumann_parts(Phi.shape, h)
    P, q = Phi.ravel(), phin.ravel()
    mu = 0.5 * Lg @ (P + q) + (P**3 + P * P * q + P * q * q + q**3) / 4
    return ((P - q) / dt - Lap @ mu).reshape(Phi.shape), mu.reshape(Phi.shape)


def neumann_mode(shape, ks, h):
    """prod_a cos(pi k_a x_a / L_a) on the cell centres: the half-wave cosines that satisfy
    the mirror condition at both walls."""
    out = 1.0
    for c, k, n in zip(inputs.cell_centres(shape, h), ks, shape):
        out = out * np.cos(math.pi * k * c / (n * h))
    return out


def neumann_kappa(ks, ns, h):
    return sum(4.0 / h**2 * math.sin(math.pi * k / (2 * n)) ** 2 for k, n in zip(ks, ns))


@pytest.mark.parametrize("shape", [(9, 12), (5, 6, 7)])
def test_neumann_operators_match_the_ghost_folded_matrices(shape):
    """Residual, J v and the assembled Jacobian with mirror walls against the hand-built
    Neumann matrices: F = (Phi - phi^n)/dt - Lap_N mu, J = I/dt - Lap_N (1/2 L_N + diag q)."""
    h = 0.8
    Phi, phin, v = rand_field(shape, 31), rand_field(shape, 32), rand_field(shape, 33, 0.0, 1.0)
    dt = 0.6
    F_ref, _ = neumann_residual_by_hand(Phi, phin, dt, h)
    F = O.residual(Phi, phin, dt, h, GAMMA, neumann=True)
    np.testing.assert_allclose(F, F_ref, rtol=0, atol=1e-12 * np.abs(F_ref).max())
    Lap, Lg = neumann_parts(shape, h)
    q = O.jac_coeff(Phi, phin).ravel()
    J_ref = np.eye(Lap.shape[0]) / dt - Lap @ (0.5 * Lg + np.diag(q))
    J = O.assemble_jacobian(Phi, phin, dt, h, GAMMA, neumann=True).toarray()
    np.testing.assert_allclose(J, J_ref, rtol=0, atol=1e-12 * np.abs(J_ref).max())
    Jv = O.jvp(v, Phi, phin, dt, h, GAMMA, neumann=True)
    np.testing.assert_allclose(Jv.ravel(), J_ref @ v.ravel(), rtol=0, atol=1e-12 * np.abs(Jv).max())
    # and they are not the periodic operators
    assert np.abs(F - O.residual(Phi, phin, dt, h, GAMMA)).max() > 1e-3 * np.abs(F).max()


@pytest.mark.parametrize("ks", [(1, 3), (2, 5)])
def test_neumann_laplacian_half_wave_symbol(ks):
    """Half-wave cosines are eigenvectors of the mirror-wall Laplacian with eigenvalue
    -sum 4/h^2 sin^2(pi k/(2N)); odd k is no mode of the periodic grid."""
    shape = (10, 12)
    h = 0.7
    u = neumann_mode(shape, ks, h)
    lam = neumann_kappa(ks, shape, h)
    np.testing.assert_allclose((neumann_lap_matrix(shape, h) @ u.ravel()).reshape(shape), -lam * u,
                               rtol=0, atol=1e-12 * lam)
    # the oracle's Jacobian at Phi = phi^n = 0 (q = 0) acts as 1/dt + kappa S/2 on the mode
    S = (1 - GAMMA) - 2 * lam + lam * lam
    zero = np.zeros(shape)
    Jv = O.jvp(u, zero, zero, 0.5, h, GAMMA, neumann=True)
    np.testing.assert_allclose(Jv, (1 / 0.5 + 0.5 * lam * S) * u, rtol=0, atol=1e-11 * (1 + lam**3))


@pytest.mark.parametrize("dt", [0.05, 1.0, 20.0])
def test_neumann_half_wave_crank_nicolson_multiplier(dt):
    """Small half-wave mode between mirror walls: one NKS step multiplies it by
    g = (1 - dt kappa S/2)/(1 + dt kappa S/2), kappa the Neumann symbol."""
    shape = (16, 16)
    h = 1.1
    ks = (1, 3)
    phi0 = 1e-6 * neumann_mode(shape, ks, h)
    lam = neumann_kappa(ks, shape, h)
    S = (1 - GAMMA) - 2 * lam + lam * lam
    g = (1 - 0.5 * dt * lam * S) / (1 + 0.5 * dt * lam * S)
    p = O.Params(parts=(2, 2), newton_rtol=1e-13, gmres_rtol=1e-12, neumann=True)
    phi1, info = O.newton_solve(phi0, dt, h, GAMMA, p)
    np.testing.assert_allclose(phi1, g * phi0, rtol=0, atol=1e-9 * 1e-6)


def test_neumann_dvd_identity_and_energy_law():
    """With mirror walls the DVD identity (Eq. DVD) and the energy balance of a step hold with
    the sums over interior edges only: F1 - F0 = -dt h^2 sum_interior (D^+ mu)^2 + dt h^2 sum mu F."""
    shape = (12, 10)
    h = 0.8
    p1, p0 = rand_field(shape, 34), rand_field(shape, 35)
    _, mu = neumann_residual_by_hand(p1, p0, 1.0, h)
    lhs = O.energy(p1, h, GAMMA, neumann=True) - O.energy(p0, h, GAMMA, neumann=True)
    assert lhs == pytest.approx(float(np.sum(mu * (p1 - p0))) * h * h, rel=1e-12)
    # the periodic energy does not satisfy it with the Neumann mu
    lhs_p = O.energy(p1, h, GAMMA) - O.energy(p0, h, GAMMA)
    assert abs(lhs_p - lhs) > 1e-6 * abs(lhs)
    phin = inputs.noise_field((16, 16), 0.07, 0.07, 36)
    dt = 1.0
    p = O.Params(parts=(2, 2), newton_rtol=1e-12, neumann=True)
    phi1, info = O.newton_solve(phin, dt, H2, GAMMA, p)
    assert info.converged
    F_by_hand, mu = neumann_residual_by_hand(phi1, phin, dt, H2)
    diss = sum(float(np.sum(np.diff(mu, axis=ax) ** 2)) / H2**2 for ax in range(2))
    F0, F1 = O.energy(phin, H2, GAMMA, neumann=True), O.energy(phi1, H2, GAMMA, neumann=True)
    assert F1 - F0 == pytest.approx(-dt * H2**2 * diss + dt * H2**2 * float(np.sum(mu * F_by_hand)),
                                    rel=1e-9, abs=1e-12 * abs(F0))
    assert F1 <= F0
    assert abs(O.mass(phi1, H2) - O.mass(phin, H2)) <= 1e-12 * max(1.0, abs(O.mass(phin, H2)))


def test_neumann_decomposition_clips_blocks_at_the_walls():
    """Cores partition the grid; overlapped blocks stop at the walls (no wrap), keep the
    overlap inside; one block is the exact inverse of the Neumann Jacobian."""
    shape, parts = (13, 10), (3, 2)
    blocks = O.decompose(shape, parts, 1, neumann=True)
    hits = np.zeros(int(np.prod(shape)), dtype=int)
    for b in blocks:
        hits[b.core_idx] += 1
        iy, ix = np.unravel_index(b.block_idx, shape)
        for c, lo, n, N in ((iy, b.core_lo[0], b.core_n[0], shape[0]), (ix, b.core_lo[1], b.core_n[1], shape[1])):
            assert c.min() == max(0, lo - 1) and c.max() == min(N - 1, lo + n)
    assert np.all(hits == 1)
    Phi, phin = rand_field(shape, 37), rand_field(shape, 38)
    J = O.assemble_jacobian(Phi, phin, 1.0, 0.8, GAMMA, neumann=True)
    pre = O.Schwarz(J, O.decompose(shape, (1, 1), 0, neumann=True), "left-ras", "lu")
    b = rand_field(shape, 39, 0.0, 1.0)
    np.testing.assert_allclose(pre.apply(b).ravel(), np.linalg.solve(J.toarray(), b.ravel()), rtol=1e-10, atol=1e-12)


def test_neumann_nks_matches_dense_direct_solve():
    """NKS step with mirror walls (clipped left-RAS blocks) against Newton with the hand-built
    Neumann residual and dense Jacobian solved by LAPACK, to 1e-12."""
    shape = (10, 9)
    phin = inputs.noise_field(shape, 0.07, 0.07, 40)
    dt = 0.5
    p = O.Params(newton_rtol=1e-13, gmres_rtol=1e-8, parts=(2, 3), overlap=1, neumann=True)
    Phi, info = O.newton_solve(phin, dt, H2, GAMMA, p)
    Lap, Lg = neumann_parts(shape, H2)
    ref = phin.copy()
    for _ in range(50):
        F, _ = neumann_residual_by_hand(ref, phin, dt, H2)
        if np.linalg.norm(F) <= 1e-14:
            break
        q = O.jac_coeff(ref, phin).ravel()
        J = np.eye(Lap.shape[0]) / dt - Lap @ (0.5 * Lg + np.diag(q))
        ref = ref - np.linalg.solve(J, F.ravel()).reshape(shape)
    assert info.converged and info.newton_its >= 2
    assert np.abs(Phi - ref).max() <= 1e-12


def test_neumann_mobility_is_conservative_and_matches_finite_differences():
    """M = 1 - phi^2 with mirror walls: sum F dt = mass change (no flux through the walls) and
    the analytic J v against central differences of F."""
    shape = (12, 10)
    Phi, phin = rand_field(shape, 41, 0.2, 0.4), rand_field(shape, 42, 0.2, 0.4)
    v = rand_field(shape, 43, 0.0, 1.0)
    dt = 0.7
    F = O.residual(Phi, phin, dt, H2, GAMMA, mobility=True, neumann=True)
    assert abs(float(np.sum(F - (Phi - phin) / dt))) <= 1e-12 * float(np.abs(F).sum())
    Jv = O.jvp(v, Phi, phin, dt, H2, GAMMA, mobility=True, neumann=True)
    eps = 1e-5 * np.linalg.norm(Phi) / np.linalg.norm(v)
    fd = (O.residual(Phi + eps * v, phin, dt, H2, GAMMA, mobility=True, neumann=True)
          - O.residual(Phi - eps * v, phin, dt, H2, GAMMA, mobility=True, neumann=True)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) <= 1e-8 * np.linalg.norm(Jv)
    J = O.assemble_jacobian(Phi, phin, dt, H2, GAMMA, mobility=True, neumann=True)
    np.testing.assert_allclose((J @ v.ravel()).reshape(shape), Jv, rtol=0, atol=1e-12 * np.abs(Jv).max())


def test_neumann_pins_catch_a_whole_cell_mirror(monkeypatch):
    """Mirroring about the wall cells (ghost u_{-1} = u_1) instead of the half-cell walls is a
    plausible mistake; the hand-built matrices catch it."""
    shape = (9, 12)
    Phi, phin = rand_field(shape, 31), rand_field(shape, 32)
    F_ref, _ = neumann_residual_by_hand(Phi, phin, 0.6, 0.8)

    def whole_cell(u):
        for ax in range(u.ndim):
            inner = np.flip(np.take(u, np.arange(1, u.shape[ax] - 1), axis=ax), axis=ax)
            u = np.concatenate([u, inner], axis=ax)
        return u

    monkeypatch.setattr(O, "even_extension", whole_cell)
    F = O.residual(Phi, phin, 0.6, 0.8, GAMMA, neumann=True)
    assert np.abs(F - F_ref).max() > 1e-3 * np.abs(F_ref).max()


# ---------------------------------------------------------------- crack propagation recipe (Test C)
def test_crack_recipe_and_first_step():
    """Test C's initial state: lattice 0.49 + cos(qy y/sqrt3) cos(qx x) - cos(2 qy y/sqrt3)/2 with
    qx = sqrt3/2, qy = 0.9 qx on the cell centres of h = pi/3 (4096 pi/3 over 4096 cells), a centred
    notch of exactly 40 x 20 cells at 0.79; one oracle step at dt_min = 1 conserves mass and lowers
    the energy."""
    w = inputs.workload("crack128x48")
    phi, h = w["phi"], w["h"]
    assert h == pytest.approx(4096 * math.pi / 3 / 4096) and w["gamma"] == 1.0
    notch = phi == 0.79
    rows, cols = np.nonzero(notch)
    assert notch.sum() == 40 * 20 and rows.min() == (48 - 20) // 2 and cols.min() == (128 - 40) // 2
    assert rows.max() - rows.min() == 19 and cols.max() - cols.min() == 39
    qx = math.sqrt(3) / 2
    qy = 0.9 * qx
    j, i = 3, 5  # a cell outside the notch
    y, x = (j + 0.5) * h, (i + 0.5) * h
    expect = 0.49 + math.cos(qy * y / math.sqrt(3)) * math.cos(qx * x) - 0.5 * math.cos(2 * qy * y / math.sqrt(3))
    assert phi[j, i] == pytest.approx(expect, rel=1e-14)
    p = O.Params(parts=w["parts"], overlap=1, dt_min=w["dt_min"], dt_max=w["dt_max"], eta=w["eta"])
    phi1, recs = O.run(phi, h, w["gamma"], p, 1)
    assert recs[0].dt == 1.0
    assert abs(recs[0].mass - O.mass(phi, h)) <= 1e-12 * abs(O.mass(phi, h))
    assert recs[0].energy < O.energy(phi, h, w["gamma"])


def test_workload_recipes_use_the_paper_parameters():
    """The crack and 3D workloads take the parameters the paper prints (tests/golden fixture with
    citations).  The 3D seed generator keeps the paper's d0, q and A; its workload runs at
    gamma = 0.3 around phi = -0.325 with four random seeds instead of the paper's 0.35 / -0.35 /
    three placed seeds: that is its stated configuration, not the paper's figure run."""
    import inspect
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_workload_parameters.json")) as f:
        g = json.load(f)
    c = g["test_c_crack"]
    assert c["domain"][0] == pytest.approx(4096 * math.pi / 3) and c["qx"] == pytest.approx(math.sqrt(3) / 2)
    w = inputs.workload("crack4096x1024")
    assert tuple(w["shape"][::-1]) == tuple(c["cells"])
    assert w["h"] * c["cells"][0] == pytest.approx(c["domain"][0]) and w["h"] * c["cells"][1] == pytest.approx(c["domain"][1])
    assert (w["gamma"], w["dt_min"], w["dt_max"], w["eta"]) == (c["gamma"], c["dt_min"], c["dt_max"], c["eta"])
    phi = w["phi"]
    assert int((phi == c["notch_value"]).sum()) == c["notch_cells"][0] * c["notch_cells"][1]
    sig = inspect.signature(inputs.crack_field).parameters
    assert sig["mean"].default == c["mean"] and sig["qx"].default == pytest.approx(c["qx"])
    assert sig["stretch"].default == c["qy_over_qx"] and sig["notch_value"].default == c["notch_value"]
    assert tuple(sig["notch_cells"].default[::-1]) == tuple(c["notch_cells"])
    d = g["test_d_bcc"]
    assert d["domain"] == pytest.approx(80 * math.pi) and d["d0"] == pytest.approx(5 * math.pi)
    sig = inspect.signature(inputs.bcc_seeds_3d).parameters
    assert sig["d0"].default == pytest.approx(d["d0"]) and sig["q"].default == pytest.approx(d["q"])
    assert sig["amp"].default == d["amplitude"]
