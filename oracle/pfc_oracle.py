"""Plain FP64 CPU oracle for one time step of the DVDM phase-field-crystal scheme,
solved by Newton-Krylov-Schwarz (Wei, Yang & Huang, arXiv:1703.01202).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct definition
the GPU path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product library never
does, and it shares no code with the CUDA path (it imports numpy/scipy only).

Conventions
-----------
* Fields are numpy float64 arrays of shape ``(Ny, Nx)`` (2D) or ``(Nz, Ny, Nx)``
  (3D); the last axis is x, so a C-order flatten gives ``idx = i + Nx*(j + Ny*k)``.
* Cell-centred periodic grid with isotropic spacing ``h`` (Sec. 3, grid
  definition x_i = (i - 1/2) dx); with ``neumann`` the grid is closed by
  Neumann-type walls (Sec. 2), as mirrors half a cell outside the end cells.
* ``gamma`` is the quench depth of Eq. (GE); mobility M = 1 (Sec. 5, tests A, B, D).

Every function cites the section / equation it follows.  Places where the paper
is silent are marked READING, each stating the reading taken.

Pinning status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, identities, brute-force dense solves); none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# --------------------------------------------------------------------------
# Difference operators (Sec. 3: D_x^+, D_x^-, D_x^<2>, Delta_d = sum of D^<2>)
# --------------------------------------------------------------------------


def d_plus(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Forward difference D^+ u = (u_{i+1} - u_i)/h, periodic (Sec. 3)."""
    return (np.roll(u, -1, axis=axis) - u) / h


def d_minus(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Backward difference D^- u = (u_i - u_{i-1})/h, periodic (Sec. 3)."""
    return (u - np.roll(u, 1, axis=axis)) / h


def d2(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Second difference D^<2> u = (u_{i+1} - 2 u_i + u_{i-1})/h^2 (Sec. 3)."""
    return (np.roll(u, -1, axis=axis) - 2.0 * u + np.roll(u, 1, axis=axis)) / (h * h)


def lap(u: np.ndarray, h: float) -> np.ndarray:
    """Discrete Laplacian Delta_d = sum over axes of D^<2> (Sec. 3); 5-point in
    2D, 7-point in 3D.  With M = 1, (div M grad)_d reduces to Delta_d."""
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        out += d2(u, ax, h)
    return out


def L_gamma(u: np.ndarray, h: float, gamma: float) -> np.ndarray:
    """Linear operator of Eq. (discretedG): [(1-gamma) + 2 Delta_d + Delta_d^2] u."""
    lu = lap(u, h)
    return (1.0 - gamma) * u + 2.0 * lu + lap(lu, h)


# --------------------------------------------------------------------------
# Discrete energy (Eq. relations, Eq. freeenergy) and mass
# --------------------------------------------------------------------------


def local_energy(phi: np.ndarray, h: float, gamma: float) -> np.ndarray:
    """Discrete local energy G_d of Eq. (relations):
    (1-g)/2 phi^2 + phi^4/4 + 1/2 (Delta_d phi)^2
      - sum over axes of [(D^+ phi)^2 + (D^- phi)^2] / 2."""
    g = 0.5 * (1.0 - gamma) * phi**2 + 0.25 * phi**4 + 0.5 * lap(phi, h) ** 2
    for ax in range(phi.ndim):
        g -= 0.5 * (d_plus(phi, ax, h) ** 2 + d_minus(phi, ax, h) ** 2)
    return g


def energy(phi: np.ndarray, h: float, gamma: float, neumann: bool = False) -> float:
    """Discrete free energy F_d = h^d * sum G_d (Eq. freeenergy); with `neumann`,
    G_d of the evenly extended field (mirror ghosts), summed over the grid."""
    if neumann:
        g = restrict_to_grid(local_energy(even_extension(phi), h, gamma), phi.shape)
        return float(np.sum(g) * h ** phi.ndim)
    return float(np.sum(local_energy(phi, h, gamma)) * h ** phi.ndim)


def mass(phi: np.ndarray, h: float) -> float:
    """Total mass h^d * sum phi, conserved by the scheme (Sec. 3, after Eq. NSOP)."""
    return float(np.sum(phi) * h ** phi.ndim)


# --------------------------------------------------------------------------
# DVD variational derivative, scheme residual, Jacobian (Eqs. discretedG, NSOP)
# --------------------------------------------------------------------------


def mu_dvd(Phi: np.ndarray, phin: np.ndarray, h: float, gamma: float) -> np.ndarray:
    """Discrete variational derivative of Eq. (discretedG):
    L_gamma (Phi + phi^n)/2 + (Phi^3 + Phi^2 phi^n + Phi phi^n^2 + phi^n^3)/4."""
    cubic = (Phi**3 + Phi**2 * phin + Phi * phin**2 + phin**3) / 4.0
    return L_gamma(0.5 * (Phi + phin), h, gamma) + cubic


# Neumann-type boundaries (Sec. 2: n . grad phi = n . grad Delta phi = n . grad Delta^2 phi = 0).
# READING: on the cell-centred grid the walls are mirrors halfway between a cell and its ghost
# (ghost phi_0 = phi_1, phi_-1 = phi_2, ...).  The field extended evenly across every wall is
# periodic on the doubled grid and stays even under every operator of the scheme, so each
# Neumann operator is the periodic one on the doubled grid, restricted back to the grid.
def even_extension(u: np.ndarray) -> np.ndarray:
    """u mirrored across the far wall of every axis: a periodic field on the doubled grid."""
    for ax in range(u.ndim):
        u = np.concatenate([u, np.flip(u, axis=ax)], axis=ax)
    return u


def restrict_to_grid(u2: np.ndarray, shape: Tuple[int, ...]) -> np.ndarray:
    return u2[tuple(slice(0, n) for n in shape)]


def mobility_nodes(Phi: np.ndarray, phin: np.ndarray) -> np.ndarray:
    """M_d of Eq. (NSOP) for M(phi) = 1 - phi^2: M at the midpoint (Phi + phi^n)/2, node by node."""
    s = 0.5 * (Phi + phin)
    return 1.0 - s * s


def div_m_grad(u: np.ndarray, Mn: np.ndarray, h: float) -> np.ndarray:
    """(div M grad)_d u = sum over axes D(M D u) (Sec. 3): the mobility on the
    midpoint of an edge is the average of its two end nodes, so the flux through
    the edge i+1/2 is (M_i + M_{i+1})/2 (u_{i+1} - u_i)/h, and the divergence is
    the difference of the fluxes through the two edges of a node, over h.  Periodic."""
    out = np.zeros_like(u)
    for ax in range(u.ndim):
        edge = 0.5 * (Mn + np.roll(Mn, -1, axis=ax))
        flux = edge * (np.roll(u, -1, axis=ax) - u) / (h * h)
        out += flux - np.roll(flux, 1, axis=ax)
    return out


def residual(Phi: np.ndarray, phin: np.ndarray, dt: float, h: float, gamma: float,
             mobility: bool = False, neumann: bool = False) -> np.ndarray:
    """Nonlinear residual of the semi-implicit scheme Eq. (NSOP):
    F(Phi) = (Phi - phi^n)/dt - (div M_d grad)_d mu(Phi, phi^n), with M = 1
    (Delta_d) or, when `mobility`, M(phi) = 1 - phi^2 evaluated at (Phi + phi^n)/2.
    READING: sign and 1/dt scaling follow the commented-out form F = (Phi -
    Phi^n)/dt + E(Phi, Phi^n) printed before Eq. (NLS).  `neumann`: the walls'
    mirror images (see even_extension)."""
    if neumann:
        return restrict_to_grid(residual(even_extension(Phi), even_extension(phin), dt, h, gamma, mobility),
                                Phi.shape)
    mu = mu_dvd(Phi, phin, h, gamma)
    if mobility:
        return (Phi - phin) / dt - div_m_grad(mu, mobility_nodes(Phi, phin), h)
    return (Phi - phin) / dt - lap(mu, h)


def jac_coeff(Phi: np.ndarray, phin: np.ndarray) -> np.ndarray:
    """q = d/dPhi of the cubic DVD term = (3 Phi^2 + 2 Phi phi^n + phi^n^2)/4."""
    return (3.0 * Phi**2 + 2.0 * Phi * phin + phin**2) / 4.0


def jvp(v: np.ndarray, Phi: np.ndarray, phin: np.ndarray, dt: float, h: float, gamma: float,
        mobility: bool = False, neumann: bool = False) -> np.ndarray:
    """Jacobian-vector product of Eq. (Jacobi): J v = v/dt - Delta_d(1/2 L_gamma v + q v).
    With `mobility` (M = 1 - phi^2 at the midpoint s = (Phi + phi^n)/2) the derivative
    of F also differentiates M_d: dM/dPhi = -2 s * 1/2 = -s, so
    J v = v/dt - (div M grad)_d(1/2 L_gamma v + q v) - (div (-s v) grad)_d mu."""
    if neumann:
        return restrict_to_grid(jvp(even_extension(v), even_extension(Phi), even_extension(phin), dt, h, gamma,
                                    mobility), v.shape)
    q = jac_coeff(Phi, phin)
    w = 0.5 * L_gamma(v, h, gamma) + q * v
    if not mobility:
        return v / dt - lap(w, h)
    s = 0.5 * (Phi + phin)
    mu = mu_dvd(Phi, phin, h, gamma)
    return v / dt - div_m_grad(w, mobility_nodes(Phi, phin), h) - div_m_grad(mu, -s * v, h)


def _lap_matrix(shape: Tuple[int, ...], h: float) -> sp.csr_matrix:
    """Assembled periodic Delta_d as a sparse matrix (C-order unknowns)."""
    n_total = int(np.prod(shape))
    out = sp.csr_matrix((n_total, n_total))
    for ax in range(len(shape)):
        n = shape[ax]
        # 1D periodic second difference along this axis.
        main = -2.0 * np.ones(n)
        d1 = sp.diags([main, np.ones(n - 1), np.ones(n - 1)], [0, 1, -1], format="lil")
        d1[0, n - 1] += 1.0
        d1[n - 1, 0] += 1.0
        d1 = d1.tocsr() / (h * h)
        left = sp.identity(int(np.prod(shape[:ax])), format="csr")
        right = sp.identity(int(np.prod(shape[ax + 1 :])), format="csr")
        out = out + sp.kron(sp.kron(left, d1), right, format="csr")
    return out.tocsr()


def _shift_matrix(shape: Tuple[int, ...], ax: int) -> sp.csr_matrix:
    """S with (S u)_i = u_{i+1} along axis ax (periodic), C-order unknowns."""
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    return sp.csr_matrix((np.ones(n), (idx.ravel(), np.roll(idx, -1, axis=ax).ravel())), shape=(n, n))


def assemble_jacobian(Phi: np.ndarray, phin: np.ndarray, dt: float, h: float, gamma: float,
                      mobility: bool = False, neumann: bool = False) -> sp.csr_matrix:
    """Assembled Jacobian J = I/dt - Delta_d (1/2 L_gamma + diag q) as CSR
    (Eq. Jacobi; L_gamma from Eq. discretedG).  With `mobility`, Delta_d becomes
    D_M = sum_ax (I - S^T) diag(M_edge) (S - I)/h^2 and the term of dM/dPhi is
    added: B = sum_ax (I - S^T) diag((S - I) mu / h^2) (I + S)/2 diag(-s).
    `neumann`: R J2 E with J2 the periodic Jacobian of the evenly extended fields on the doubled
    grid, E the even extension (grid -> doubled grid) and R the restriction."""
    if neumann:
        shape = Phi.shape
        n = Phi.size
        src = even_extension(np.arange(n).reshape(shape)).ravel()
        E = sp.csr_matrix((np.ones(src.size), (np.arange(src.size), src)), shape=(src.size, n))
        J2 = assemble_jacobian(even_extension(Phi), even_extension(phin), dt, h, gamma, mobility)
        rows = np.ravel_multi_index(np.indices(shape).reshape(len(shape), -1), tuple(2 * m for m in shape))
        Rsel = sp.csr_matrix((np.ones(n), (np.arange(n), rows)), shape=(n, J2.shape[0]))
        J = (Rsel @ J2 @ E).tocsr()
        J.sum_duplicates()
        return J
    shape = Phi.shape
    n = Phi.size
    lapm = _lap_matrix(shape, h)
    eye = sp.identity(n, format="csr")
    lg = (1.0 - gamma) * eye + 2.0 * lapm + lapm @ lapm
    q = sp.diags(jac_coeff(Phi, phin).ravel())
    if not mobility:
        J = eye / dt - lapm @ (0.5 * lg + q)
    else:
        Mn = mobility_nodes(Phi, phin).ravel()
        mu = mu_dvd(Phi, phin, h, gamma).ravel()
        s = 0.5 * (Phi + phin).ravel()
        DM = sp.csr_matrix((n, n))
        B = sp.csr_matrix((n, n))
        for ax in range(len(shape)):
            S = _shift_matrix(shape, ax)
            edge = 0.5 * (Mn + S @ Mn)
            DM = DM + (eye - S.T) @ sp.diags(edge) @ (S - eye) / (h * h)
            grad_mu = (S @ mu - mu) / (h * h)
            B = B + (eye - S.T) @ sp.diags(grad_mu) @ (0.5 * (eye + S)) @ sp.diags(-s)
        J = eye / dt - DM @ (0.5 * lg + q) - B
    J = J.tocsr()
    J.sum_duplicates()
    return J


# --------------------------------------------------------------------------
# Overlapping decomposition and Schwarz preconditioners (Sec. 4, Eqs. invM, ras, ash, Ak)
# --------------------------------------------------------------------------


def split_axis(n: int, p: int) -> List[Tuple[int, int]]:
    """Even split of n cells into p cores; the first (n mod p) cores get one
    extra cell.  READING: the paper only says 'np non-overlapping subdomains'."""
    base, extra = divmod(n, p)
    out, start = [], 0
    for r in range(p):
        size = base + (1 if r < extra else 0)
        out.append((start, size))
        start += size
    return out


@dataclass
class Block:
    """One subdomain: the core Omega_k and the overlapped block Omega_k^delta."""

    core_lo: Tuple[int, ...]  # per-axis start of the core (array axis order)
    core_n: Tuple[int, ...]  # per-axis core size
    overlap: int
    shape: Tuple[int, ...]  # global grid shape
    neumann: bool = False  # walls instead of periodic wrap: the block is clipped to the grid
    dims: Tuple[int, ...] = field(default=None)  # per-axis extent of Omega_k^delta (clipped at walls)
    block_idx: np.ndarray = field(default=None)  # global flat indices of Omega_k^delta (block C-order)
    core_mask: np.ndarray = field(default=None)  # True where the block point is in Omega_k
    core_idx: np.ndarray = field(default=None)  # global flat indices of Omega_k (block order)

    def __post_init__(self):
        axes = []
        masks = []
        for lo, n, N in zip(self.core_lo, self.core_n, self.shape):
            if n + 2 * self.overlap > N and not self.neumann:  # between walls the block is clipped
                raise ValueError("block wider than the periodic grid")
            if self.neumann:  # READING: at a wall the overlapped block stops at the wall
                a0, a1 = max(0, lo - self.overlap), min(N, lo + n + self.overlap)
                axes.append(np.arange(a0, a1))
                m = np.zeros(a1 - a0, dtype=bool)
                m[lo - a0 : lo - a0 + n] = True
            else:
                axes.append(np.arange(lo - self.overlap, lo + n + self.overlap) % N)
                m = np.zeros(n + 2 * self.overlap, dtype=bool)
                m[self.overlap : self.overlap + n] = True
            masks.append(m)
        self.dims = tuple(len(ax) for ax in axes)
        grids = np.meshgrid(*axes, indexing="ij")
        self.block_idx = np.ravel_multi_index(tuple(g.ravel() for g in grids), self.shape)
        mg = np.meshgrid(*masks, indexing="ij")
        self.core_mask = np.logical_and.reduce([m.ravel() for m in mg])
        self.core_idx = self.block_idx[self.core_mask]


def decompose(shape: Tuple[int, ...], parts: Tuple[int, ...], overlap: int, neumann: bool = False) -> List[Block]:
    """Non-overlapping cores Omega_k extended by `overlap` cells per side with
    periodic wrap (Sec. 4), or clipped at the walls with Neumann-type boundaries.
    `parts` is given in array-axis order."""
    splits = [split_axis(N, p) for N, p in zip(shape, parts)]
    blocks = []
    for combo in np.ndindex(*parts):
        lo = tuple(splits[a][combo[a]][0] for a in range(len(shape)))
        n = tuple(splits[a][combo[a]][1] for a in range(len(shape)))
        blocks.append(Block(lo, n, overlap, tuple(shape), neumann))
    return blocks


def subdomain_matrix(J: sp.csr_matrix, blk: Block) -> np.ndarray:
    """A_k = R_k^delta J (R_k^delta)^T (Eq. Ak) as a dense matrix."""
    idx = blk.block_idx
    return J[idx][:, idx].toarray()


def subdomain_matrix_improved_bc(
    Phi: np.ndarray, phin: np.ndarray, dt: float, h: float, gamma: float, blk: Block
) -> np.ndarray:
    """A_k from the discretised subdomain problem with phi = 0 on the 3-layer ring
    Omega_k^{delta+1} minus Omega_k^delta (Sec. 4, 'improved' boundary condition):
    column c is the local operator applied to the c-th unit vector of the block,
    on a local grid that is the block plus a zero ring of width 3 (the stencil
    radius of Delta_d L_gamma).  q is taken from the global fields."""
    ring = 3
    ext_shape = tuple(n + 2 * blk.overlap + 2 * ring for n in blk.core_n)
    # global coordinates of the extended local grid (periodic wrap)
    axes = [
        np.arange(lo - blk.overlap - ring, lo + n + blk.overlap + ring) % N
        for lo, n, N in zip(blk.core_lo, blk.core_n, blk.shape)
    ]
    q_glob = jac_coeff(Phi, phin)
    q_loc = q_glob[np.ix_(*axes)]
    inner = tuple(slice(ring, ring + n + 2 * blk.overlap) for n in blk.core_n)

    def lap_zero(u):
        # Laplacian on the local grid; values beyond the local grid never
        # reach the block rows (ring width 3 = stencil radius), so zero
        # padding is exact there.
        out = np.zeros_like(u)
        for ax in range(u.ndim):
            up = np.zeros_like(u)
            dn = np.zeros_like(u)
            sl_a = [slice(None)] * u.ndim
            sl_b = [slice(None)] * u.ndim
            sl_a[ax] = slice(0, -1)
            sl_b[ax] = slice(1, None)
            up[tuple(sl_a)] = u[tuple(sl_b)]
            dn[tuple(sl_b)] = u[tuple(sl_a)]
            out += (up + dn - 2.0 * u) / (h * h)
        return out

    nb = int(np.prod([n + 2 * blk.overlap for n in blk.core_n]))
    A = np.zeros((nb, nb))
    unit = np.zeros(ext_shape)
    for c in range(nb):
        unit[...] = 0.0
        unit[inner].flat[c] = 1.0
        lv = lap_zero(unit)
        lgv = (1.0 - gamma) * unit + 2.0 * lv + lap_zero(lv)
        col = unit / dt - lap_zero(0.5 * lgv + q_loc * unit)
        A[:, c] = col[inner].ravel()
    return A


def block_pattern(blk: Block, radius: int = 3) -> np.ndarray:
    """Structural pattern of A_k: block points whose local offsets satisfy
    |d|_1 <= 3, the support of Delta_d (1/2 L_gamma + q) (radius-3 composed stencil)."""
    dims = blk.dims
    coords = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, len(dims))
    dist = np.abs(coords[:, None, :] - coords[None, :, :]).sum(-1)
    return dist <= radius


def ilu0(A: sp.csr_matrix) -> sp.csr_matrix:
    """ILU(0) of a sparse matrix, natural row order, fill restricted to the
    pattern of A (Sec. 4 / Sec. 5.2: the 3D subdomain solver).  Row-oriented
    (IKJ) Gaussian elimination: for each row i and each k < i in row i's
    pattern, a_ik /= a_kk and a_ij -= a_ik a_kj for j > k in both patterns.
    Returns one CSR holding L (unit lower, strict part) and U (upper incl. diag)."""
    return ilu0_batch([A])[0]


def ilu0_batch(mats: Sequence[sp.csr_matrix]) -> List[sp.csr_matrix]:
    """ilu0 of several matrices with one sparsity pattern (the blocks of one extent),
    factored side by side: the same elimination steps, in the same order, on each
    matrix's values (a stacked array, one row per matrix)."""
    As = [sp.csr_matrix(A, dtype=np.float64, copy=True) for A in mats]
    for A in As:
        A.sort_indices()
    indptr, indices = As[0].indptr, As[0].indices
    for A in As[1:]:
        if not (np.array_equal(A.indptr, indptr) and np.array_equal(A.indices, indices)):
            raise ValueError("ilu0_batch: the matrices must share one pattern")
    n = As[0].shape[0]
    D = np.stack([A.data for A in As])  # D[b, p]: entry p of matrix b
    pos = [dict(zip(indices[indptr[i] : indptr[i + 1]], range(indptr[i], indptr[i + 1]))) for i in range(n)]
    diag_pos = np.array([pos[i][i] for i in range(n)])
    for i in range(n):
        row = pos[i]
        for p in range(indptr[i], indptr[i + 1]):
            k = indices[p]
            if k >= i:
                break
            D[:, p] /= D[:, diag_pos[k]]  # l_ik = a_ik / a_kk
            upper = range(diag_pos[k] + 1, indptr[k + 1])  # a_kj, j > k
            pairs = [(row[indices[pk]], pk) for pk in upper if indices[pk] in row]
            if pairs:
                pj, pk = (np.array(v) for v in zip(*pairs))
                D[:, pj] -= D[:, p : p + 1] * D[:, pk]  # a_ij -= l_ik a_kj (distinct j: independent)
    for b, A in enumerate(As):
        A.data = D[b].copy()
    return As


def ilu0_split(LU: sp.csr_matrix) -> Tuple[sp.csr_matrix, sp.csr_matrix]:
    """The unit lower factor L (with its unit diagonal) and the upper factor U of an ILU(0)."""
    L = sp.tril(LU, -1, format="csr") + sp.identity(LU.shape[0], format="csr")
    return L, sp.triu(LU, 0, format="csr")


def ilu0_solve(LU: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """Forward substitution with the unit lower factor, then backward
    substitution with the upper factor of an ILU(0) (library triangular solves)."""
    return ilu0_split_solve(ilu0_split(LU), b)


def ilu0_split_solve(LU: Tuple[sp.csr_matrix, sp.csr_matrix], b: np.ndarray) -> np.ndarray:
    L, U = LU
    y = spla.spsolve_triangular(L, b, lower=True, unit_diagonal=True)
    return spla.spsolve_triangular(U, y, lower=False)


class Schwarz:
    """Additive Schwarz preconditioners of Sec. 4:
    kind 'as'        : sum_k (R_k^delta)^T inv(A_k) R_k^delta   (Eq. invM)
    kind 'left-ras'  : sum_k (R_k^0)^T     inv(A_k) R_k^delta   (Eq. ras)
    kind 'right-ras' : sum_k (R_k^delta)^T inv(A_k) R_k^0       (Eq. ash)
    Subdomain solver: dense LU with partial pivoting ('lu') or ILU(0) ('ilu0').
    READING (3D): ILU(0) of the 63-point block matrices breaks down (negative
    pivots) at the 3D workload's time steps, so 'ilu0' factors A_k + sigma I with
    sigma = ilu_shift * mean |diag A_k| (a shifted incomplete factorisation);
    ilu_shift = 0 is plain ILU(0)."""

    def __init__(self, J: sp.csr_matrix, blocks: Sequence[Block], kind: str = "left-ras", solver: str = "lu",
                 ilu_shift: float = 0.0):
        if kind not in ("as", "left-ras", "right-ras"):
            raise ValueError(kind)
        self.blocks = list(blocks)
        self.kind = kind
        self.solver = solver
        self.factors = [None] * len(self.blocks)
        if solver == "lu":
            for k, blk in enumerate(self.blocks):
                self.factors[k] = scipy.linalg.lu_factor(subdomain_matrix(J, blk), check_finite=True)
        elif solver == "ilu0":
            by_extent = {}  # blocks of one extent share their pattern: factored together
            for k, blk in enumerate(self.blocks):
                by_extent.setdefault(blk.dims, []).append(k)
            self.groups = []  # (block numbers, block-diagonal L, block-diagonal U) per extent
            for ks in by_extent.values():
                pattern = block_pattern(self.blocks[ks[0]])
                rows, cols = np.nonzero(pattern)
                mats = []
                for k in ks:
                    A = subdomain_matrix(J, self.blocks[k])
                    if np.any(A[~pattern] != 0.0):
                        raise ValueError("block couples to itself across the periodic wrap; grid too small")
                    A = A + ilu_shift * np.mean(np.abs(np.diag(A))) * np.eye(A.shape[0])
                    mats.append(sp.csr_matrix((A[rows, cols], (rows, cols)), shape=A.shape))
                for k, LU in zip(ks, ilu0_batch(mats)):
                    self.factors[k] = ilu0_split(LU)
                # the blocks' triangular systems side by side: one block-diagonal solve per extent
                # visits every block's rows and entries in the order its own solve would
                self.groups.append((ks, sp.block_diag([self.factors[k][0] for k in ks], format="csr"),
                                    sp.block_diag([self.factors[k][1] for k in ks], format="csr")))
        else:
            raise ValueError(solver)

    def _solve(self, k: int, rhs: np.ndarray) -> np.ndarray:
        if self.solver == "lu":
            return scipy.linalg.lu_solve(self.factors[k], rhs)
        return ilu0_split_solve(self.factors[k], rhs)

    def _solve_all(self, rhs: List[np.ndarray]) -> List[np.ndarray]:
        if self.solver == "lu":
            return [self._solve(k, b) for k, b in enumerate(rhs)]
        sols = [None] * len(rhs)
        for ks, L, U in self.groups:
            y = spla.spsolve_triangular(L, np.concatenate([rhs[k] for k in ks]), lower=True, unit_diagonal=True)
            x = spla.spsolve_triangular(U, y, lower=False)
            o = 0
            for k in ks:
                sols[k] = x[o : o + rhs[k].size]
                o += rhs[k].size
        return sols

    def apply(self, r: np.ndarray) -> np.ndarray:
        flat = r.ravel()
        z = np.zeros_like(flat)
        rhs = []
        for blk in self.blocks:
            b = flat[blk.block_idx]
            if self.kind == "right-ras":
                b = np.where(blk.core_mask, b, 0.0)  # restriction R_k^0
            rhs.append(b)
        for k, (blk, sol) in enumerate(zip(self.blocks, self._solve_all(rhs))):
            if self.kind == "left-ras":
                z[blk.core_idx] += sol[blk.core_mask]  # extension (R_k^0)^T
            else:
                np.add.at(z, blk.block_idx, sol)  # extension (R_k^delta)^T
        return z.reshape(r.shape)


# --------------------------------------------------------------------------
# Right-preconditioned restarted GMRES (Sec. 4, Eq. hjacobi)
# --------------------------------------------------------------------------


@dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    residual_estimate: float
    converged: bool


def gmres_right(
    matvec: Callable[[np.ndarray], np.ndarray],
    precond: Callable[[np.ndarray], np.ndarray],
    b: np.ndarray,
    tol: float,
    restart: int = 30,
    max_it: int = 10000,
) -> GmresResult:
    """GMRES on J H^{-1} (H S) = b (Eq. hjacobi), x0 = 0, modified Gram-Schmidt
    Arnoldi, Givens rotations for the least-squares problem, stop when the
    least-squares residual estimate <= tol.  S = x0 + sum_j y_j H^{-1} v_j.
    READING: restart length and orthogonalisation are not given in the paper."""
    x = np.zeros_like(b)
    its = 0
    beta = float(np.linalg.norm(b))
    if beta <= tol:
        return GmresResult(x, 0, beta, True)
    r = b.copy()
    while its < max_it:
        beta = float(np.linalg.norm(r))
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        est = beta
        for j in range(restart):
            z = precond(V[j])
            w = matvec(z)
            Z.append(z)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = float(np.vdot(V[i].ravel(), w.ravel()))
                w = w - H[i, j] * V[i]
            hnext = float(np.linalg.norm(w))
            H[j + 1, j] = hnext
            for i in range(j):  # apply the previous rotations to column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            denom = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / denom
            sn[j] = H[j + 1, j] / denom
            H[j, j] = denom
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            est = abs(g[j + 1])
            if est <= tol or its >= max_it or hnext == 0.0:
                break
            V.append(w / hnext)
        # back substitution on the rotated Hessenberg system
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1 : j_done] @ y[i + 1 : j_done]) / H[i, i]
        for i in range(j_done):
            x = x + y[i] * Z[i]
        if est <= tol or its >= max_it:
            return GmresResult(x, its, est, est <= tol)
        r = b - matvec(x)  # restart
    return GmresResult(x, its, est, False)


# --------------------------------------------------------------------------
# Inexact Newton with line search (Sec. 4, Eqs. newton, Jacobi, stop test)
# --------------------------------------------------------------------------


@dataclass
class Params:
    """Solver parameters.  Defaults are the settings the workloads here run with (Newton
    rtol 1e-10, GMRES rtol 1e-6, left-RAS); the paper's own are eps_r = 1e-8,
    eps_a = 1e-10, xi_r = 1e-3, xi_a = 1e-11 (Sec. 5)."""

    newton_rtol: float = 1e-10
    newton_atol: float = 0.0
    newton_max_it: int = 50
    gmres_rtol: float = 1e-6
    gmres_atol: float = 0.0
    gmres_restart: int = 30
    gmres_max_it: int = 10000
    parts: Tuple[int, ...] = (4, 4)  # subdomains per array axis
    overlap: int = 1  # cells added per side (READING of '3 delta layers')
    ras_kind: str = "left-ras"
    subdomain_solver: str = "lu"  # 'lu' (2D) or 'ilu0' (3D)
    ilu_shift: float = 0.1  # READING: relative diagonal shift of the 3D ILU(0) blocks
    precond: bool = True  # False: H = I
    mass_projection: bool = True  # READING: zero-mean Newton update
    ls_alpha: float = 1e-4  # Armijo constant of the backtracking line search
    ls_max_cuts: int = 10
    dt_min: float = 1e-2
    dt_max: float = 10.0
    eta: float = 5000.0
    energy_scaled: bool = True  # READING: controller uses F_d / |Omega|
    dt_halvings: int = 0  # READING: a step whose Newton iteration fails is retried with dt / 2
    mobility: bool = False  # M(phi) = 1 - phi^2 (Eq. NSOP's M_d); False: M = 1
    neumann: bool = False  # Neumann-type walls (Sec. 2) instead of the periodic grid


@dataclass
class StepInfo:
    newton_its: int
    gmres_its: int
    res_norm0: float
    res_norm: float
    lambdas: List[float]
    converged: bool


def newton_solve(
    phin: np.ndarray, dt: float, h: float, gamma: float, p: Params, guess: Optional[np.ndarray] = None,
    ref_norm: Optional[float] = None,
) -> Tuple[np.ndarray, StepInfo]:
    """One time step: solve F(Phi) = 0 (Eq. NLS) by inexact Newton (Eq. newton)
    Phi_{m+1} = Phi_m + lambda_m S_m, with S_m from right-preconditioned GMRES
    on J_m S_m = -F(Phi_m) (Eqs. Jacobi, hjacobi), stopping when
    ||F(Phi_{m+1})|| <= max(eps_r ||F(Phi_0)||, eps_a).  Initial guess: phi^n
    (Sec. 4) unless `guess` is given.  The Schwarz factors are built once per
    step at the first Newton iteration and reused (Sec. 5.2, factor reuse).
    READING: with another initial guess the tolerance stays the plain method's,
    eps_r ||F(phi^n)|| (`ref_norm`), so a better guess cannot tighten it.

    READINGS: 2-norms throughout; backtracking line search on f = ||F||^2/2 with
    the Armijo test f(Phi + lam S) <= (1 - 2 alpha lam) f(Phi) and quadratic
    backtracking lam <- clamp(lam^2 f0 / (f(lam) - f0 + 2 lam f0) ... ) to
    [0.1 lam, 0.5 lam]; optional projection of S to zero mean (mass)."""
    Phi = (phin if guess is None else guess).copy()
    F = residual(Phi, phin, dt, h, gamma, p.mobility, p.neumann)
    r0 = float(np.linalg.norm(F))
    target = max(p.newton_rtol * (r0 if ref_norm is None else ref_norm), p.newton_atol)
    rnorm = r0
    m = 0
    gm_total = 0
    lambdas: List[float] = []
    pre = None
    while rnorm > target and m < p.newton_max_it:
        J = assemble_jacobian(Phi, phin, dt, h, gamma, p.mobility, p.neumann)
        if p.precond and pre is None:
            pre = Schwarz(J, decompose(Phi.shape, p.parts, p.overlap, p.neumann), p.ras_kind, p.subdomain_solver,
                          p.ilu_shift)
        precond = (lambda v: pre.apply(v)) if p.precond else (lambda v: v)
        matvec = lambda v: (J @ v.ravel()).reshape(v.shape)
        res = gmres_right(
            matvec, precond, -F, max(p.gmres_rtol * rnorm, p.gmres_atol), p.gmres_restart, p.gmres_max_it
        )
        gm_total += res.iterations
        S = res.x
        if p.mass_projection:
            S = S - np.mean(S)
        f0 = 0.5 * rnorm * rnorm
        lam = 1.0
        for cut in range(p.ls_max_cuts + 1):
            trial = Phi + lam * S
            Ft = residual(trial, phin, dt, h, gamma, p.mobility, p.neumann)
            ft = 0.5 * float(np.dot(Ft.ravel(), Ft.ravel()))
            if ft <= (1.0 - 2.0 * p.ls_alpha * lam) * f0 or cut == p.ls_max_cuts:
                break
            # minimiser of the quadratic through f0, slope -2 f0, f(lam)
            lam_q = lam * lam * f0 / (ft - f0 + 2.0 * lam * f0)
            lam = min(max(lam_q, 0.1 * lam), 0.5 * lam)
        lambdas.append(lam)
        Phi, F = trial, Ft
        rnorm = float(np.linalg.norm(F))
        m += 1
    return Phi, StepInfo(m, gm_total, r0, rnorm, lambdas, rnorm <= target)


# --------------------------------------------------------------------------
# Adaptive time step (Eq. sencondt) and the time loop
# --------------------------------------------------------------------------


def adaptive_dt(E_n: float, E_nm1: float, dt_prev: float, p: Params) -> float:
    """dt_n = max(dt_min, dt_max / sqrt(1 + eta |F'|^2)), F' = (E^n - E^{n-1})/dt_{n-1}
    (Eq. sencondt).  E is F_d, or F_d/|Omega| when p.energy_scaled (READING)."""
    fp = (E_n - E_nm1) / dt_prev
    return max(p.dt_min, p.dt_max / math.sqrt(1.0 + p.eta * fp * fp))


def extrapolated_guess(phin: np.ndarray, phinm1: np.ndarray, dt: float, dt_prev: float) -> np.ndarray:
    """Linear extrapolation phi^n + (dt/dt_prev)(phi^n - phi^{n-1}) (initial-guess
    alternative; the paper's own guess is phi^n, Sec. 4)."""
    return phin + (dt / dt_prev) * (phin - phinm1)


@dataclass
class RunRecord:
    t: float
    dt: float
    energy: float
    mass: float
    newton_its: int
    gmres_its: int


def _step_with_guess(phin, phinm1, dt, dt_prev, h, gamma, p, guess):
    """One Newton solve from phi^n or, for guess == "extrap", the safeguarded extrapolation."""
    if guess == "extrap" and dt_prev is not None:
        # READING (safeguard): the extrapolation is used only when its residual norm
        # is not larger than that of phi^n, the paper's own starting point (Sec. 4);
        # after a step-size jump dt/dt_prev is large and the extrapolation poor.
        g = extrapolated_guess(phin, phinm1, dt, dt_prev)
        ref = float(np.linalg.norm(residual(phin, phin, dt, h, gamma, p.mobility, p.neumann)))
        if ref < np.linalg.norm(residual(g, phin, dt, h, gamma, p.mobility, p.neumann)):
            g = None
        return newton_solve(phin, dt, h, gamma, p, g, ref_norm=ref)
    return newton_solve(phin, dt, h, gamma, p, None)


def run(
    phi0: np.ndarray,
    h: float,
    gamma: float,
    p: Params,
    nsteps: int,
    fixed_dt: Optional[float] = None,
    guess: str = "prev",
) -> Tuple[np.ndarray, List[RunRecord]]:
    """Time loop.  With fixed_dt None, dt follows Eq. (sencondt); the first step
    uses dt_min (READING: the paper does not say how the controller starts)."""
    area = h ** phi0.ndim * phi0.size
    scale = 1.0 / area if p.energy_scaled else 1.0
    phin = phi0.copy()
    phinm1 = phi0.copy()
    E_n = energy(phin, h, gamma, p.neumann)
    E_nm1 = None
    dt_prev = None
    t = 0.0
    recs: List[RunRecord] = []
    for n in range(nsteps):
        if fixed_dt is not None:
            dt = fixed_dt
        elif E_nm1 is None:
            dt = p.dt_min
        else:
            dt = adaptive_dt(E_n * scale, E_nm1 * scale, dt_prev, p)
        for cut in range(p.dt_halvings + 1):
            phi1, info = _step_with_guess(phin, phinm1, dt, dt_prev, h, gamma, p, guess)
            if info.converged:
                break
            dt *= 0.5
        if not info.converged:
            raise RuntimeError(f"Newton did not converge at step {n}")
        phinm1, phin = phin, phi1
        E_nm1, E_n = E_n, energy(phin, h, gamma, p.neumann)
        dt_prev = dt
        t += dt
        recs.append(RunRecord(t, dt, E_n, mass(phin, h), info.newton_its, info.gmres_its))
    return phin, recs
