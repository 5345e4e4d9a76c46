"""The C-ABI library builds, loads without a GPU, and exports every entry point
declared in include/*.h; host-side validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpfc():
    from paper_1703_01202_gb300 import build, pfc

    build.build()
    return pfc.lib()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(pfc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(libpfc):
    names = declared_functions()
    assert "pfc_step" in names and "pfc_create" in names
    for n in names:
        assert hasattr(libpfc, n), n


def test_binding_covers_header():
    from paper_1703_01202_gb300 import pfc

    bound = {n for n, _, _ in pfc._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_struct_sizes_match_c_layout(libpfc):
    from paper_1703_01202_gb300 import pfc

    # pfc_params filled by the library round-trips through the ctypes mirror
    p = pfc.default_params()
    assert p.newton_rtol == 1e-10 and p.gmres_rtol == 1e-6 and p.gmres_restart == 30
    assert p.ras_kind == pfc.PFC_LEFT_RAS and p.overlap == 1 and p.eta == 5000.0 and p.energy_scaled == 1


def test_workspace_size_and_validation(libpfc):
    from paper_1703_01202_gb300 import pfc

    p = pfc.default_params(sub=(64, 64), overlap=1)
    size = pfc.workspace_size((1024, 1024), p)
    # 11 fields + 31 + 30 Krylov vectors of 8 MiB plus the F64 band factors of 4096 blocks
    assert size > (11 + 61) * 8 * 1024 * 1024
    with pytest.raises(pfc.PfcError) as e:
        pfc.workspace_size((16, 16), pfc.default_params(sub=(1, 1), overlap=1))  # 16 + 2 > 16
    assert e.value.status == pfc.PFC_EINVAL
    with pytest.raises(pfc.PfcError):
        pfc.workspace_size((64, 64), pfc.default_params(sub=(4, 4), gmres_restart=0))
    # 3D grids have two apply kernels (0: global memory, 1: shared-memory window); 2..5 are 2D ones
    for v in (-1, 0, 1):
        assert pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2), apply_variant=v)) > 0
    for v in (2, 5):
        with pytest.raises(pfc.PfcError):
            pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2), apply_variant=v))
    assert pfc.status_str(pfc.PFC_ESINGULAR).startswith("zero pivot")


def test_schwarz_kind_validation(libpfc):
    """AS and right-RAS take the chunked apply on 2D grids (plus one scratch row of n_max
    doubles per block for the overlap sums); 3D grids and the per-step launch shapes refuse them."""
    from paper_1703_01202_gb300 import pfc

    left = pfc.workspace_size((1024, 1024), pfc.default_params(sub=(64, 64), overlap=1))
    for kind in (pfc.PFC_AS, pfc.PFC_RIGHT_RAS):
        size = pfc.workspace_size((1024, 1024), pfc.default_params(sub=(64, 64), overlap=1, ras_kind=kind))
        assert size >= left + 4096 * 324 * 8
        assert pfc.workspace_size((1024, 1024), pfc.default_params(sub=(64, 64), ras_kind=kind, apply_variant=5)) == size
        for bad in (dict(apply_variant=0), dict(apply_variant=4)):
            with pytest.raises(pfc.PfcError) as e:
                pfc.workspace_size((1024, 1024), pfc.default_params(sub=(64, 64), ras_kind=kind, **bad))
            assert e.value.status == pfc.PFC_EINVAL
        with pytest.raises(pfc.PfcError) as e:
            pfc.workspace_size((64, 64, 64), pfc.default_params(sub=(4, 4, 4), ras_kind=kind))
        assert e.value.status == pfc.PFC_EINVAL
    with pytest.raises(pfc.PfcError):
        pfc.workspace_size((64, 64), pfc.default_params(sub=(4, 4), ras_kind=7))


def test_mobility_validation(libpfc):
    """M = 1 - phi^2 (mobility = 1): 2D and 3D periodic grids; four more fields in the workspace
    (mu and the midpoint s beside q and the trial q)."""
    from paper_1703_01202_gb300 import pfc

    base = pfc.workspace_size((64, 64), pfc.default_params(sub=(4, 4)))
    assert pfc.workspace_size((64, 64), pfc.default_params(sub=(4, 4), mobility=1)) >= base + 4 * 64 * 64 * 8
    for bad in (dict(mobility=2), dict(mobility=-1)):
        with pytest.raises(pfc.PfcError):
            pfc.workspace_size((64, 64), pfc.default_params(sub=(4, 4), **bad))
    base3 = pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2)))
    assert pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2), mobility=1)) >= base3 + 4 * 32 ** 3 * 8


def test_boundary_validation(libpfc):
    """Neumann-type walls (boundary = 1): at least 4 cells per axis (2D and 3D), left-RAS, M = 1;
    3D blocks at least 7 cells per axis (a block at a wall has one overlap)."""
    from paper_1703_01202_gb300 import pfc

    assert pfc.workspace_size((64, 48), pfc.default_params(sub=(4, 4), boundary=pfc.PFC_NEUMANN)) > 0
    for shape, bad in (((64, 64), dict(boundary=2)), ((64, 64), dict(boundary=-1)),
                       ((64, 64), dict(boundary=1, ras_kind=pfc.PFC_AS, apply_variant=5)),
                       ((64, 64), dict(boundary=1, mobility=1)), ((3, 64), dict(boundary=1, sub=(1, 1), overlap=0))):
        prm = dict(sub=(4, 4))
        prm.update(bad)
        with pytest.raises(pfc.PfcError):
            pfc.workspace_size(shape, pfc.default_params(**prm))
    assert pfc.workspace_size((3, 64), pfc.default_params(sub=(1, 1), overlap=0)) > 0  # periodic: fine
    assert pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2), boundary=1)) > 0
    assert pfc.workspace_size((8, 8, 8), pfc.default_params(sub=(1, 1, 1), overlap=0, boundary=1)) > 0
    for shape, sub in (((10, 10, 10), (2, 2, 2)),  # wall blocks of 5 + 1 cells
                       ((6, 6, 6), (1, 1, 1))):    # a block of 6 cells per axis
        with pytest.raises(pfc.PfcError):
            pfc.workspace_size(shape, pfc.default_params(sub=sub, overlap=1 if sub[0] > 1 else 0, boundary=1))
    with pytest.raises(pfc.PfcError):
        pfc.workspace_size((32, 32, 32), pfc.default_params(sub=(2, 2, 2), boundary=1, mobility=1))


def test_static_residual_and_wait_selftest_validation(libpfc):
    """Arguments both entry points refuse before any device work (so no GPU is needed):
    the static residual takes pfc_create's grid and scalar checks; the wait self-test
    its flag and cycle-limit range."""
    from paper_1703_01202_gb300 import pfc

    L = libpfc
    one = ctypes.c_void_p(8)  # never dereferenced: every call below fails validation first
    nrm = ctypes.c_double()

    def static(shape, h=0.78, eps=0.25, dt=1.0):
        g = pfc.make_grid(shape)
        return L.pfc_residual_static(ctypes.byref(g), h, eps, one, one, dt, one, ctypes.byref(nrm), None)

    g3 = pfc.make_grid((4, 4))
    g3.n[2] = 2  # a 2D grid with two planes
    assert L.pfc_residual_static(ctypes.byref(g3), 0.78, 0.25, one, one, 1.0, one, None, None) == pfc.PFC_EINVAL
    for kw in (dict(h=float("inf")), dict(h=0.0), dict(eps=float("inf")), dict(eps=float("nan")),
               dict(dt=float("inf")), dict(dt=-1.0)):
        assert static((64, 64), **kw) == pfc.PFC_EINVAL, kw
    assert static((8, 8, 8)) == pfc.PFC_EINVAL
    assert static((8192, 8192)) == pfc.PFC_EINVAL  # more tiles than the fixed scratch holds
    assert L.pfc_wait_selftest(0, 1000, None, None) == pfc.PFC_EINVAL
    assert L.pfc_wait_selftest(2, 1000, one, None) == pfc.PFC_EINVAL
    assert L.pfc_wait_selftest(0, 0, one, None) == pfc.PFC_EINVAL
    assert L.pfc_wait_selftest(0, 5_000_000_000, one, None) == pfc.PFC_EINVAL
