"""Host logic of the subdomain decomposition (Sec. 4) through the C ABI, without a GPU:
the blocks the library factors (pfc_block_layout) against the oracle's decomposition, cell
by cell and in the same order, for periodic grids (wrapping blocks), Neumann walls (blocks
clipped at the walls), uneven splits, overlaps 0-3 and 3D."""
import numpy as np
import pytest

from oracle import pfc_oracle as O


@pytest.fixture(scope="module")
def pfc():
    from paper_1703_01202_gb300 import build, pfc as P

    build.build()
    P.lib()
    return P


def cells(row, shape):
    """Global flat indices of a block and of its core, block-local C order, from one layout row."""
    nd = len(shape)
    lo, ext, off, core = row[0:3], row[3:6], row[6:9], row[9:12]
    # layout rows are x-first; the grid shape is in array-axis order (last axis x)
    axes, caxes = [], []
    for a in range(nd):
        xa = nd - 1 - a  # layout component of array axis a
        n = shape[a]
        ax = (lo[xa] + np.arange(ext[xa])) % n
        axes.append(ax)
        caxes.append(ax[off[xa]: off[xa] + core[xa]])
    blk = np.ravel_multi_index(tuple(g.ravel() for g in np.meshgrid(*axes, indexing="ij")), shape)
    cor = np.ravel_multi_index(tuple(g.ravel() for g in np.meshgrid(*caxes, indexing="ij")), shape)
    return blk, cor


CASES = [((64, 64), (4, 4), 1, 0), ((37, 50), (3, 7), 1, 0), ((50, 37), (3, 2), 2, 0), ((21, 27), (3, 3), 3, 0),
         ((16, 16), (2, 2), 0, 0), ((64, 64), (4, 4), 1, 1), ((37, 50), (3, 7), 1, 1), ((50, 37), (3, 2), 2, 1),
         ((21, 27), (3, 3), 3, 1), ((9, 13), (1, 1), 0, 1), ((25, 20, 18), (2, 2, 2), 1, 0)]


@pytest.mark.parametrize("shape,parts,overlap,neumann", CASES)
def test_block_layout_matches_the_oracle_decomposition(pfc, shape, parts, overlap, neumann):
    params = pfc.default_params(sub=tuple(parts[::-1]), overlap=overlap, boundary=neumann)
    rows = pfc.block_layout(shape, params)
    ref = O.decompose(shape, parts, overlap, neumann=bool(neumann))
    assert len(rows) == len(ref)
    for row, b in zip(rows, ref):
        blk, cor = cells(row, shape)
        np.testing.assert_array_equal(blk, b.block_idx)
        np.testing.assert_array_equal(cor, b.core_idx)
        if neumann:  # no wrap between walls
            assert row[0] >= 0 and row[1] >= 0
            assert row[0] + row[3] <= shape[-1] and row[1] + row[4] <= shape[-2]


def test_block_layout_errors(pfc):
    params = pfc.default_params(sub=(4, 4))
    with pytest.raises(pfc.PfcError):
        pfc.block_layout((64, 64), pfc.default_params(sub=(4, 4), boundary=1, mobility=1))
    grid = pfc.make_grid((64, 64))
    import ctypes

    n = ctypes.c_int(0)
    assert pfc.lib().pfc_block_layout(ctypes.byref(grid), ctypes.byref(params), None, 1, ctypes.byref(n)) \
        == pfc.PFC_EINVAL
    assert pfc.lib().pfc_block_layout(ctypes.byref(grid), ctypes.byref(params), None, 0, None) == pfc.PFC_EINVAL
    assert pfc.lib().pfc_block_layout(ctypes.byref(grid), ctypes.byref(params), None, 0, ctypes.byref(n)) \
        == pfc.PFC_OK and n.value == 16
