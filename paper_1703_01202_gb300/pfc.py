"""ctypes binding of libpfc (include/pfc.h).

Argument marshalling only: every numeric step runs in the CUDA kernels of
libpfc.so.  PyTorch supplies the device workspace and the stream.  The library
is loaded on first use; if it is missing or fails to load, the call raises --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int64, c_longlong, c_size_t, c_void_p
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfc.so")

PFC_OK, PFC_EINVAL, PFC_ENOMEM, PFC_ECUDA = 0, -1, -2, -3
PFC_ENEWTON, PFC_EGMRES, PFC_ESINGULAR, PFC_ENAN, PFC_ETIMEOUT = -4, -5, -6, -7, -8
PFC_F64, PFC_F32, PFC_BF16 = 0, 1, 2
PFC_AS, PFC_LEFT_RAS, PFC_RIGHT_RAS = 0, 1, 2
PFC_PERIODIC, PFC_NEUMANN = 0, 1  # pfc_params.boundary
PFC_GUESS_PREV, PFC_GUESS_EXTRAP, PFC_GUESS_USER, PFC_GUESS_LEARNED = 0, 1, 2, 3
N_APPLY_VARIANTS = 6  # apply kernels 0-4 (per-step solves, bitwise equal) and 5 (chunked solves)
APPLY_CHUNKED = 5


class pfc_grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int64 * 3)]


class pfc_params(ctypes.Structure):
    _fields_ = [
        ("newton_rtol", c_double), ("newton_atol", c_double), ("newton_max_it", c_int),
        ("gmres_rtol", c_double), ("gmres_atol", c_double), ("gmres_restart", c_int), ("gmres_max_it", c_int),
        ("sub", c_int * 3), ("overlap", c_int), ("ras_kind", c_int), ("factor_prec", c_int), ("guess", c_int),
        ("mass_projection", c_int), ("ls_alpha", c_double), ("ls_max_cuts", c_int),
        ("dt_min", c_double), ("dt_max", c_double), ("eta", c_double), ("energy_scaled", c_int),
        ("apply_variant", c_int), ("dt_halvings", c_int), ("gmres_reorth_eta", c_double),
        ("use_graph", c_int), ("reuse_factor", c_int), ("mobility", c_int), ("boundary", c_int),
        ("gmres_fast_dots", c_int), ("jvp_fp32", c_int),
    ]


class pfc_step_info(ctypes.Structure):
    _fields_ = [
        ("status", c_int), ("newton_its", c_int), ("gmres_its", c_int), ("ls_cuts", c_int),
        ("dt", c_double), ("energy", c_double), ("mass", c_double), ("res_norm0", c_double), ("res_norm", c_double),
        ("guess_used", c_int), ("dt_cuts", c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pfc_kernel_prof(ctypes.Structure):
    _fields_ = [("launches", c_longlong), ("ms", c_double), ("bytes", c_double), ("flops", c_double),
                ("bytes_stored", c_double)]


PROF_KINDS = ["apply", "jvp", "dot", "axpy", "factor", "residual", "records"]  # PFC_PROF_* order


class PfcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


# (name, restype, argtypes) of every entry point declared in include/pfc.h
_SIGNATURES = [
    ("pfc_default_params", c_int, [POINTER(pfc_params)]),
    ("pfc_workspace_size", c_int, [POINTER(pfc_grid), POINTER(pfc_params), POINTER(c_size_t)]),
    ("pfc_block_layout", c_int, [POINTER(pfc_grid), POINTER(pfc_params), c_void_p, c_int, POINTER(c_int)]),
    ("pfc_create", c_int, [POINTER(pfc_grid), c_double, c_double, POINTER(pfc_params), c_void_p, c_size_t, c_void_p,
                           POINTER(c_void_p)]),
    ("pfc_destroy", None, [c_void_p]),
    ("pfc_set_field", c_int, [c_void_p, c_void_p, c_int]),
    ("pfc_get_field", c_int, [c_void_p, c_void_p, c_int]),
    ("pfc_set_guess", c_int, [c_void_p, c_void_p, c_int]),
    ("pfc_step", c_int, [c_void_p, c_double, POINTER(pfc_step_info)]),
    ("pfc_run", c_int, [c_void_p, c_int, POINTER(pfc_step_info)]),
    ("pfc_energy", c_int, [c_void_p, POINTER(c_double)]),
    ("pfc_mass", c_int, [c_void_p, POINTER(c_double)]),
    ("pfc_residual", c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, POINTER(c_double)]),
    ("pfc_jvp", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_void_p]),
    ("pfc_precond_apply", c_int, [c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
    ("pfc_next_dt", c_int, [c_void_p, POINTER(c_double)]),
    ("pfc_step_host", c_int, [c_void_p, c_void_p, c_double, c_void_p, POINTER(pfc_step_info)]),
    ("pfc_profile", c_int, [c_void_p, c_int]),
    ("pfc_save", c_int, [c_void_p, c_char_p]),
    ("pfc_load", c_int, [c_void_p, c_char_p]),
    ("pfc_run_batch", c_int, [POINTER(c_void_p), c_int, c_int, c_void_p, POINTER(c_int)]),
    ("pfc_get_tuning", c_int, [c_void_p, POINTER(c_int), POINTER(c_float), POINTER(c_int)]),
    ("pfc_profile_read", c_int, [c_void_p, POINTER(c_longlong), POINTER(c_double), POINTER(c_double),
                                 POINTER(c_longlong)]),
    ("pfc_profile_kernels", c_int, [c_void_p, POINTER(pfc_kernel_prof), c_int]),
    ("pfc_launch_counts", c_int, [POINTER(c_longlong), POINTER(c_longlong)]),
    ("pfc_residual_static", c_int, [POINTER(pfc_grid), c_double, c_double, c_void_p, c_void_p, c_double, c_void_p,
                                    POINTER(c_double), c_void_p]),
    ("pfc_wait_selftest", c_int, [c_int, c_longlong, c_void_p, c_void_p]),
    ("pfc_cnn_param_count", c_int, []),
    ("pfc_cnn_workspace_size", c_int, [c_int64, c_int64, POINTER(c_size_t)]),
    ("pfc_cnn_create", c_int, [c_int64, c_int64, c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]),
    ("pfc_cnn_destroy", None, [c_void_p]),
    ("pfc_cnn_set_params", c_int, [c_void_p, c_void_p]),
    ("pfc_cnn_get_params", c_int, [c_void_p, c_void_p]),
    ("pfc_cnn_forward", c_int, [c_void_p, c_void_p, c_void_p]),
    ("pfc_cnn_loss_grad", c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    ("pfc_cnn_train_step", c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_double)]),
    ("pfc_cnn_sample", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_double, c_void_p,
                               c_void_p]),
    ("pfc_set_guess_net", c_int, [c_void_p, c_void_p, c_double]),
    ("pfc_status_str", c_char_p, [c_int]),
]

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libpfc.so (raises if it is absent: build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpfc.so not built ({LIB_PATH}); run paper_1703_01202_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(st: int) -> str:
    try:
        return lib().pfc_status_str(st).decode()
    except Exception:
        return "unknown"


def _check(st: int, what: str):
    if st != PFC_OK:
        raise PfcError(st, what)


def default_params(**over) -> pfc_params:
    p = pfc_params()
    _check(lib().pfc_default_params(ctypes.byref(p)), "pfc_default_params")
    for k, v in over.items():
        if k == "sub":
            for a, s in enumerate(v):
                p.sub[a] = int(s)
        elif any(k == f for f, _ in pfc_params._fields_):
            setattr(p, k, v)
        else:
            raise KeyError(f"pfc_params has no field {k!r}")
    return p


def run_batch(solvers: Sequence["Solver"], nsteps: int) -> List[List[dict]]:
    """pfc_run_batch over independent solvers (create each on its own stream so
    their kernels overlap); returns the per-step records of every solver."""
    n = len(solvers)
    handles = (c_void_p * n)(*[s.handle.value for s in solvers])
    infos = (pfc_step_info * max(n * nsteps, 1))()
    status = (c_int * n)()
    st = lib().pfc_run_batch(handles, n, int(nsteps), ctypes.cast(infos, c_void_p), status)
    out = [[infos[i * nsteps + k].as_dict() for k in range(nsteps)] for i in range(n)]
    _check(st, "pfc_run_batch")
    return out


def launch_counts() -> dict:
    """Process-wide: kernels the library has run and CUDA graph launches."""
    k, g = c_longlong(), c_longlong()
    _check(lib().pfc_launch_counts(ctypes.byref(k), ctypes.byref(g)), "pfc_launch_counts")
    return {"kernels": k.value, "graphs": g.value}


def make_grid(shape: Sequence[int]) -> pfc_grid:
    """Grid from an array shape in array-axis order ((Ny, Nx) or (Nz, Ny, Nx))."""
    g = pfc_grid()
    g.dim = len(shape)
    rev = list(shape)[::-1]
    for a in range(3):
        g.n[a] = int(rev[a]) if a < len(rev) else 1
    return g


def workspace_size(shape: Sequence[int], params: pfc_params) -> int:
    out = c_size_t(0)
    _check(lib().pfc_workspace_size(ctypes.byref(make_grid(shape)), ctypes.byref(params), ctypes.byref(out)),
           "pfc_workspace_size")
    return out.value


def block_layout(shape: Sequence[int], params: pfc_params) -> np.ndarray:
    """The subdomains a state factors (host only): an (nblocks, 12) int32 array of rows
    x0, y0, z0, bx, by, bz, ox, oy, oz, cx, cy, cz in the library's block order."""
    count = c_int(0)
    grid = make_grid(shape)
    _check(lib().pfc_block_layout(ctypes.byref(grid), ctypes.byref(params), None, 0, ctypes.byref(count)),
           "pfc_block_layout")
    out = np.zeros((count.value, 12), dtype=np.int32)
    _check(lib().pfc_block_layout(ctypes.byref(grid), ctypes.byref(params), out.ctypes.data_as(c_void_p),
                                  count.value, ctypes.byref(count)), "pfc_block_layout")
    return out


class Solver:
    """One PFC state on the current CUDA device: a thin owner of the workspace
    (a torch uint8 tensor) and of the pfc_state handle."""

    def __init__(self, shape: Sequence[int], h: float, gamma: float, params: Optional[pfc_params] = None,
                 stream=None, device: str = "cuda"):
        import torch

        self.torch = torch
        self.shape = tuple(int(s) for s in shape)
        self.n = int(np.prod(self.shape))
        self.params = params if params is not None else default_params()
        self.grid = make_grid(self.shape)
        size = workspace_size(self.shape, self.params)
        self.device = torch.device(device)
        self.ws = torch.empty(max(size, 256), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        handle = c_void_p()
        _check(lib().pfc_create(ctypes.byref(self.grid), float(h), float(gamma), ctypes.byref(self.params),
                                c_void_p(self.ws.data_ptr()), c_size_t(self.ws.numel()),
                                c_void_p(self.stream.cuda_stream), ctypes.byref(handle)), "pfc_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().pfc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- fields
    def _dev(self, x):
        t = self.torch
        if isinstance(x, np.ndarray):
            x = t.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(self.device)
        assert x.dtype == t.float64 and x.is_cuda and x.is_contiguous() and x.numel() == self.n
        return x

    def set_field(self, phi):
        if isinstance(phi, np.ndarray):
            a = np.ascontiguousarray(phi, dtype=np.float64)
            assert a.size == self.n
            _check(lib().pfc_set_field(self.handle, a.ctypes.data_as(c_void_p), 0), "pfc_set_field")
        else:
            d = self._dev(phi)
            _check(lib().pfc_set_field(self.handle, c_void_p(d.data_ptr()), 1), "pfc_set_field")

    def save(self, path: str):
        _check(lib().pfc_save(self.handle, os.fsencode(path)), "pfc_save")

    def load(self, path: str):
        _check(lib().pfc_load(self.handle, os.fsencode(path)), "pfc_load")

    def get_field(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        _check(lib().pfc_get_field(self.handle, out.ctypes.data_as(c_void_p), 0), "pfc_get_field")
        return out

    def get_field_device(self, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self.shape, dtype=t.float64, device=self.device)
        _check(lib().pfc_get_field(self.handle, c_void_p(out.data_ptr()), 1), "pfc_get_field")
        return out

    def set_guess(self, guess):
        if isinstance(guess, np.ndarray):
            a = np.ascontiguousarray(guess, dtype=np.float64)
            _check(lib().pfc_set_guess(self.handle, a.ctypes.data_as(c_void_p), 0), "pfc_set_guess")
        else:
            d = self._dev(guess)
            _check(lib().pfc_set_guess(self.handle, c_void_p(d.data_ptr()), 1), "pfc_set_guess")

    # -- stepping
    def step(self, dt: float) -> dict:
        info = pfc_step_info()
        _check(lib().pfc_step(self.handle, float(dt), ctypes.byref(info)), "pfc_step")
        return info.as_dict()

    def run(self, nsteps: int) -> List[dict]:
        infos = (pfc_step_info * max(nsteps, 1))()
        st = lib().pfc_run(self.handle, int(nsteps), infos)
        out = [infos[i].as_dict() for i in range(nsteps)]
        _check(st, "pfc_run")
        return out

    def energy(self) -> float:
        v = c_double()
        _check(lib().pfc_energy(self.handle, ctypes.byref(v)), "pfc_energy")
        return v.value

    def mass(self) -> float:
        v = c_double()
        _check(lib().pfc_mass(self.handle, ctypes.byref(v)), "pfc_mass")
        return v.value

    def next_dt(self) -> float:
        v = c_double()
        _check(lib().pfc_next_dt(self.handle, ctypes.byref(v)), "pfc_next_dt")
        return v.value

    def step_host(self, phin_host: np.ndarray, dt: float, out_host: np.ndarray) -> dict:
        """One step through host buffers (float64, C-contiguous; pinned memory recommended)."""
        assert phin_host.dtype == np.float64 and out_host.dtype == np.float64
        assert phin_host.flags.c_contiguous and out_host.flags.c_contiguous
        info = pfc_step_info()
        _check(lib().pfc_step_host(self.handle, phin_host.ctypes.data_as(c_void_p), float(dt),
                                   out_host.ctypes.data_as(c_void_p), ctypes.byref(info)), "pfc_step_host")
        return info.as_dict()

    def profile(self, enable: bool):
        _check(lib().pfc_profile(self.handle, 1 if enable else 0), "pfc_profile")

    def profile_read(self) -> dict:
        a, k = c_longlong(), c_longlong()
        ms, b = c_double(), c_double()
        _check(lib().pfc_profile_read(self.handle, ctypes.byref(a), ctypes.byref(ms), ctypes.byref(b),
                                      ctypes.byref(k)), "pfc_profile_read")
        return {"apply_launches": a.value, "apply_ms": ms.value, "apply_bytes": b.value, "kernel_launches": k.value}

    def profile_kernels(self) -> dict:
        """Per kernel family (PROF_KINDS): timed launches, summed ms, algorithmic bytes and flops,
        and the bytes of the storage format in use, since profiling was enabled."""
        arr = (pfc_kernel_prof * len(PROF_KINDS))()
        _check(lib().pfc_profile_kernels(self.handle, arr, len(PROF_KINDS)), "pfc_profile_kernels")
        return {name: {k: getattr(arr[i], k) for k, _ in pfc_kernel_prof._fields_}
                for i, name in enumerate(PROF_KINDS)}

    def tuning(self) -> dict:
        v, gr = c_int(), c_int()
        ms = (c_float * N_APPLY_VARIANTS)()
        _check(lib().pfc_get_tuning(self.handle, ctypes.byref(v), ms, ctypes.byref(gr)), "pfc_get_tuning")
        return {"apply_variant": v.value, "apply_ms": [ms[i] for i in range(N_APPLY_VARIANTS)], "graph": gr.value}

    # -- test hooks on device tensors
    def residual(self, Phi, phin, dt: float):
        t = self.torch
        P, N = self._dev(Phi), self._dev(phin)
        F = t.empty(self.shape, dtype=t.float64, device=self.device)
        nrm = c_double()
        _check(lib().pfc_residual(self.handle, c_void_p(P.data_ptr()), c_void_p(N.data_ptr()), float(dt),
                                  c_void_p(F.data_ptr()), ctypes.byref(nrm)), "pfc_residual")
        return F, nrm.value

    def jvp(self, Phi, phin, v, dt: float):
        t = self.torch
        P, N, V = self._dev(Phi), self._dev(phin), self._dev(v)
        out = t.empty(self.shape, dtype=t.float64, device=self.device)
        _check(lib().pfc_jvp(self.handle, c_void_p(P.data_ptr()), c_void_p(N.data_ptr()), c_void_p(V.data_ptr()),
                             float(dt), c_void_p(out.data_ptr())), "pfc_jvp")
        return out

    def precond_apply(self, Phi, phin, dt: float, r):
        t = self.torch
        P, N, R = self._dev(Phi), self._dev(phin), self._dev(r)
        out = t.zeros(self.shape, dtype=t.float64, device=self.device)
        _check(lib().pfc_precond_apply(self.handle, c_void_p(P.data_ptr()), c_void_p(N.data_ptr()), float(dt),
                                       c_void_p(R.data_ptr()), c_void_p(out.data_ptr())), "pfc_precond_apply")
        return out


class GuessNet:
    """The learned-initial-guess network on one grid (workspace owned by a torch tensor)."""

    def __init__(self, shape: Sequence[int], stream=None, device: str = "cuda"):
        import torch

        self.torch = torch
        self.shape = tuple(int(s) for s in shape)
        assert len(self.shape) == 2
        ny, nx = self.shape
        self.n = nx * ny
        size = c_size_t(0)
        _check(lib().pfc_cnn_workspace_size(nx, ny, ctypes.byref(size)), "pfc_cnn_workspace_size")
        self.device = torch.device(device)
        self.ws = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = c_void_p()
        _check(lib().pfc_cnn_create(nx, ny, c_void_p(self.ws.data_ptr()), c_size_t(self.ws.numel()),
                                    c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "pfc_cnn_create")
        self.handle = h

    @staticmethod
    def param_count() -> int:
        return lib().pfc_cnn_param_count()

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().pfc_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta: np.ndarray):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.param_count()
        _check(lib().pfc_cnn_set_params(self.handle, a.ctypes.data_as(c_void_p)), "pfc_cnn_set_params")

    def get_params(self) -> np.ndarray:
        a = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().pfc_cnn_get_params(self.handle, a.ctypes.data_as(c_void_p)), "pfc_cnn_get_params")
        return a

    def forward(self, feat):
        """feat: device float64 tensor (3, ny, nx); returns (ny, nx) float64."""
        t = self.torch
        out = t.empty(self.shape, dtype=t.float64, device=self.device)
        _check(lib().pfc_cnn_forward(self.handle, c_void_p(feat.data_ptr()), c_void_p(out.data_ptr())),
               "pfc_cnn_forward")
        return out

    def loss_grad(self, feat, target):
        g = np.empty(self.param_count(), dtype=np.float32)
        loss = c_double()
        _check(lib().pfc_cnn_loss_grad(self.handle, c_void_p(feat.data_ptr()), c_void_p(target.data_ptr()),
                                       ctypes.byref(loss), g.ctypes.data_as(c_void_p)), "pfc_cnn_loss_grad")
        return loss.value, g

    def sample(self, phinm1, phin, phinp1, r: float, c2: float, s_out: float, feat, target):
        """Fills feat (3, ny, nx) and target (ny, nx) device tensors from three consecutive fields."""
        _check(lib().pfc_cnn_sample(self.handle, c_void_p(phinm1.data_ptr()), c_void_p(phin.data_ptr()),
                                    c_void_p(phinp1.data_ptr()), float(r), float(c2), float(s_out),
                                    c_void_p(feat.data_ptr()), c_void_p(target.data_ptr())), "pfc_cnn_sample")

    def train_step(self, feat, target, lr: float, t: int, want_loss: bool = True) -> float:
        loss = c_double(float("nan"))
        _check(lib().pfc_cnn_train_step(self.handle, c_void_p(feat.data_ptr()), c_void_p(target.data_ptr()),
                                        float(lr), int(t), ctypes.byref(loss) if want_loss else None),
               "pfc_cnn_train_step")
        return loss.value


def set_guess_net(solver: "Solver", net: Optional[GuessNet], s_out: float):
    _check(lib().pfc_set_guess_net(solver.handle, net.handle if net is not None else None, float(s_out)),
           "pfc_set_guess_net")
