"""B300 HAMLS: harmonic approximation on S^2 via moving least squares.

A thin ctypes binding over the C ABI in ``include/hamls.h`` (and the
inspection calls of ``include/hamls_debug.h``). It only marshals arguments:
every step of the method runs in the CUDA library ``libhamls.so``, which must
have been built (``python -m paper_2609_39200_b300.build`` or
``__graft_entry__.build()``). There is no fallback: if the library cannot be
loaded, importing the binding raises.

PyTorch provides device memory and streams. Arrays may be torch tensors (on
the GPU or pinned/pageable host memory) or numpy arrays (host); host inputs
are copied by the library on the plan's stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhamls.so")

HAMLS_FP64, HAMLS_MIXED = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "cuda error", 4: "underdetermined",
          5: "support too large", 6: "timeout", 7: "non-finite value", 8: "capacity exceeded",
          9: "voronoi cell failed"}
STAGES = ("cells", "aux_knn", "shepard", "order", "stage_values", "mls", "fft", "legendre", "voronoi")


class HamlsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("n_target", ctypes.c_int), ("eps", ctypes.c_double), ("chi_target", ctypes.c_double),
                ("chi_full", ctypes.c_double), ("sobolev_s", ctypes.c_double), ("aux_points", ctypes.c_int64),
                ("aux_radius", ctypes.c_double), ("pivot_floor", ctypes.c_double), ("precision", ctypes.c_int),
                ("fp64_pivot", ctypes.c_double), ("weight_fn", ctypes.c_int)]


class FitStats(ctypes.Structure):
    _fields_ = [("sum_n", ctypes.c_int64), ("min_n", ctypes.c_int64), ("max_n", ctypes.c_int64),
                ("n_regularized", ctypes.c_int64), ("n_guarded", ctypes.c_int64), ("n_fp64_redo", ctypes.c_int64),
                ("n_dropped", ctypes.c_int64), ("grid_nodes", ctypes.c_int64), ("aux_points", ctypes.c_int64),
                ("bands", ctypes.c_int32), ("cells", ctypes.c_int32), ("knn_candidates", ctypes.c_int64),
                ("knn_scans", ctypes.c_int64),
                ("knn_exact_fallbacks", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "hamls_default_params": (None, [ctypes.POINTER(Params)]),
    "hamls_plan": (_I, [ctypes.POINTER(_P), _P, _P, _I64, _I, _I, ctypes.POINTER(Params), _P]),
    "hamls_replan": (_I, [_P, _P, _P, _I64, _P]),
    "hamls_plan_reserve": (_I, [ctypes.POINTER(_P), _I64, _I, _I, ctypes.POINTER(Params), _P]),
    "hamls_plan_footprint": (_I, [_I64, _I, _I, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "hamls_fit": (_I, [_P, _P, _P, _P]),
    "hamls_forward": (_I, [_P, _P, _P, _I64, _P, _P]),
    "hamls_quadrature_batch": (_I, [_P, _P, _P, _I, _P]),
    "hamls_refit_prepare": (_I, [_P, _P]),
    "hamls_refit": (_I, [_P, _P, _P, _P]),
    "hamls_refit_batch": (_I, [_P, _P, _P, _I, _P]),
    "hamls_voronoi_areas": (_I, [_P, _P, _P]),
    "hamls_voronoi_weights": (_I, [_P, _P]),
    "hamls_sync": (_I, [_P, _I]),
    "hamls_status_async": (_I, [_P, _P, _P]),
    "hamls_status_from_flags": (_I, [ctypes.c_uint32]),
    "hamls_stats": (_I, [_P, ctypes.POINTER(FitStats)]),
    "hamls_destroy": (_I, [_P]),
    "hamls_status_string": (ctypes.c_char_p, [_I]),
    "hamls_set_timing": (_I, [_P, _I]),
    "hamls_stage_times": (_I, [_P, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(_I)]),
    "hamls_launch_count": (_I64, [_P, _I]),
    "hamls_debug_cells": (_I, [_P, _P, _P, _P, _P]),
    "hamls_debug_knn": (_I, [_P, _P, _I64, _I, _P, _P]),
    "hamls_debug_ball": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "hamls_debug_grid": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "hamls_debug_aux": (_I, [_P, _P, _P, _P]),
    "hamls_debug_quadrature": (_I, [_P, _P, _P, _P]),
    "hamls_debug_gl": (_I, [_P, _P, _P, _P]),
    "hamls_cells_noalloc": (_I, [_P, _I64, _I, _I, _P, _P, _P, _P]),
    "hamls_debug_tc_gemm": (_I, [_P, _P, _P, _I, _I, _I, _P]),
}
EXPORTS = tuple(_SIGS)

_lib = None


def lib() -> ctypes.CDLL:
    """Load libhamls.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_params(**kw) -> Params:
    p = Params()
    lib().hamls_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": HAMLS_FP64, "mixed": HAMLS_MIXED}[v]
        setattr(p, k, v)
    return p


def _check(code: int, where: str):
    if code != 0:
        raise HamlsError(code, where)


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "array must be C-contiguous"
        return a.ctypes.data
    raise TypeError(type(a))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def n_coeffs(N: int) -> int:
    return (N + 1) * (N + 2) // 2


class Plan:
    """A HAMLS plan: nodes x_i (M x 3 float64 unit vectors), bandwidth N, degree K."""

    def __init__(self, nodes, N: int, K: int, weights=None, params: Optional[Params] = None, stream=None,
                 capacity: Optional[int] = None, **kw):
        """A plan for ``nodes`` (hamls_plan); with nodes=None, a plan reserved
        for up to ``capacity`` nodes that a replan fills (hamls_plan_reserve)."""
        self.N, self.K = int(N), int(K)
        self.params = params if params is not None else default_params(**kw)
        h = ctypes.c_void_p()
        if nodes is None:
            self.M, self.capacity = 0, int(capacity)
            self._keep = None
            _check(lib().hamls_plan_reserve(ctypes.byref(h), self.capacity, self.N, self.K,
                                            ctypes.byref(self.params), _stream(stream)), "hamls_plan_reserve")
        else:
            self.M = int(nodes.shape[0])
            self.capacity = self.M
            self._keep = (nodes, weights)
            _check(lib().hamls_plan(ctypes.byref(h), _ptr(nodes), _ptr(weights), self.M, self.N, self.K,
                                    ctypes.byref(self.params), _stream(stream)), "hamls_plan")
        self.h = h

    @property
    def mixed(self) -> bool:
        return self.params.precision == HAMLS_MIXED

    def replan(self, nodes, weights=None, stream=None):
        self._keep = (nodes, weights)
        M = int(nodes.shape[0])
        _check(lib().hamls_replan(self.h, _ptr(nodes), _ptr(weights), M, _stream(stream)), "hamls_replan")
        self.M = M

    def fit(self, values, out=None, stream=None):
        """Coefficients as a float64 tensor (ncoef, 2) = (re, im), packed m-major.
        ``out`` may be a device tensor or pinned host tensor of that shape."""
        if out is None:
            dev = values.device if isinstance(values, torch.Tensor) and values.is_cuda else torch.device("cuda")
            out = torch.empty((n_coeffs(self.N), 2), dtype=torch.float64, device=dev)
        self._keep_fit = (values, out)
        _check(lib().hamls_fit(self.h, _ptr(values), _ptr(out), _stream(stream)), "hamls_fit")
        return out

    def forward(self, coeffs, points=None, out=None, stream=None):
        """The forward transform (hamls_forward): values of the real field
        with these coefficients ((ncoef, 2) float64) at the plan's nodes
        (points=None; node order of the last plan/replan) or at points
        ((P, 3) float64 device tensor); float64 tensor of the values."""
        if points is None:
            n = self.M
            if out is None:
                out = torch.empty(n, dtype=torch.float64, device="cuda")
        else:
            n = int(points.shape[0])
            if out is None:
                out = torch.empty(n, dtype=torch.float64, device=points.device)
        self._keep_fwd = (coeffs, points, out)
        _check(lib().hamls_forward(self.h, _ptr(coeffs), _ptr(points), n, _ptr(out), _stream(stream)),
               "hamls_forward")
        return out

    def quadrature_batch(self, fgrid, out=None, stream=None):
        """Step 3 for B sets of grid values (B x M_Q float64 device tensor):
        coefficients (B, ncoef, 2), on the tensor cores for mixed plans."""
        B = int(fgrid.shape[0])
        if out is None:
            out = torch.empty((B, n_coeffs(self.N), 2), dtype=torch.float64, device=fgrid.device)
        self._keep_qb = (fgrid, out)
        _check(lib().hamls_quadrature_batch(self.h, _ptr(fgrid), _ptr(out), B, _stream(stream)),
               "hamls_quadrature_batch")
        return out

    def refit_prepare(self, stream=None):
        """Keep the fit for the current nodes as a sparse operator of the values."""
        _check(lib().hamls_refit_prepare(self.h, _stream(stream)), "hamls_refit_prepare")

    def refit(self, values, out=None, stream=None):
        """Coefficients for new values at the prepared nodes (same layout as fit)."""
        if out is None:
            dev = values.device if isinstance(values, torch.Tensor) and values.is_cuda else torch.device("cuda")
            out = torch.empty((n_coeffs(self.N), 2), dtype=torch.float64, device=dev)
        self._keep_refit = (values, out)
        _check(lib().hamls_refit(self.h, _ptr(values), _ptr(out), _stream(stream)), "hamls_refit")
        return out

    def refit_batch(self, values, out=None, stream=None):
        """Coefficients (B, ncoef, 2) for B value sets (B x M float64 device
        tensor) at the prepared nodes."""
        B = int(values.shape[0])
        if out is None:
            out = torch.empty((B, n_coeffs(self.N), 2), dtype=torch.float64, device=values.device)
        self._keep_rb = (values, out)
        _check(lib().hamls_refit_batch(self.h, _ptr(values), _ptr(out), B, _stream(stream)), "hamls_refit_batch")
        return out

    def voronoi_areas(self, out=None, stream=None):
        """Areas of the spherical Voronoi cells of the plan's nodes (M float64,
        node order). ``out`` may be a device tensor or a host tensor."""
        if out is None:
            out = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self._keep_vor = out
        _check(lib().hamls_voronoi_areas(self.h, _ptr(out), _stream(stream)), "hamls_voronoi_areas")
        return out

    def voronoi_weights(self, stream=None):
        """Use the Voronoi areas of the current nodes as the weights v_i."""
        _check(lib().hamls_voronoi_weights(self.h, _stream(stream)), "hamls_voronoi_weights")

    def status_async(self, flags, stream=None):
        """Enqueue a copy of the device status word into ``flags`` (a uint32
        slot: an int32 tensor element on the device or in pinned host memory)
        and clear it; read it once the stream has passed this point and map
        it with ``status_from_flags``."""
        _check(lib().hamls_status_async(self.h, _ptr(flags), _stream(stream)), "hamls_status_async")

    def sync(self, timeout_ms: int = -1):
        _check(lib().hamls_sync(self.h, int(timeout_ms)), "hamls_sync")

    def stats(self) -> dict:
        s = FitStats()
        _check(lib().hamls_stats(self.h, ctypes.byref(s)), "hamls_stats")
        return s.as_dict()

    def set_timing(self, on: bool = True):
        _check(lib().hamls_set_timing(self.h, 1 if on else 0), "hamls_set_timing")

    def stage_times(self) -> dict:
        buf = (ctypes.c_float * 16)()
        n = ctypes.c_int()
        _check(lib().hamls_stage_times(self.h, buf, 16, ctypes.byref(n)), "hamls_stage_times")
        return {STAGES[i]: buf[i] for i in range(n.value)}

    def launch_count(self, reset: bool = False) -> int:
        return int(lib().hamls_launch_count(self.h, 1 if reset else 0))

    # ---------------------------------------------------------------- debug
    def debug_cells(self, stream=None):
        st = self.stats()
        dev = torch.device("cuda")
        keys = torch.empty(self.M, dtype=torch.int32, device=dev)
        perm = torch.empty(self.M, dtype=torch.int32, device=dev)
        start = torch.empty(st["bands"] * st["cells"] + 1, dtype=torch.int32, device=dev)
        _check(lib().hamls_debug_cells(self.h, _ptr(keys), _ptr(perm), _ptr(start), _stream(stream)),
               "hamls_debug_cells")
        return keys, perm, start, st["bands"], st["cells"]

    def debug_knn(self, queries: torch.Tensor, n: int, stream=None) -> torch.Tensor:
        out = torch.empty(queries.shape[0], dtype=torch.float64, device=queries.device)
        _check(lib().hamls_debug_knn(self.h, _ptr(queries), queries.shape[0], int(n), _ptr(out), _stream(stream)),
               "hamls_debug_knn")
        return out

    def debug_ball(self, queries: torch.Tensor, rho2: torch.Tensor, stream=None):
        nq = queries.shape[0]
        dev = queries.device
        cnt = torch.empty(nq, dtype=torch.int64, device=dev)
        ids = torch.empty(nq, dtype=torch.int64, device=dev)
        hx = torch.empty(nq, dtype=torch.int64, device=dev)
        _check(lib().hamls_debug_ball(self.h, _ptr(queries), _ptr(rho2), nq, _ptr(cnt), _ptr(ids), _ptr(hx),
                                      _stream(stream)), "hamls_debug_ball")
        return cnt, ids, hx

    def debug_grid(self, stream=None) -> dict:
        MQ = (self.N + 1) * (2 * self.N + 2)
        dev = torch.device("cuda")
        d = {k: torch.empty(MQ, dtype=torch.float64, device=dev) for k in ("delta", "chi", "tau", "f")}
        cnt = torch.empty(MQ, dtype=torch.int32, device=dev)
        _check(lib().hamls_debug_grid(self.h, _ptr(d["delta"]), _ptr(cnt), _ptr(d["chi"]), _ptr(d["tau"]),
                                      _ptr(d["f"]), _stream(stream)), "hamls_debug_grid")
        d["count"] = cnt
        return d

    def debug_aux(self, stream=None):
        st = self.stats()
        dev = torch.device("cuda")
        xyz = torch.empty((st["aux_points"], 3), dtype=torch.float64, device=dev)
        dn = torch.empty(st["aux_points"], dtype=torch.float64, device=dev)
        _check(lib().hamls_debug_aux(self.h, _ptr(xyz), _ptr(dn), _stream(stream)), "hamls_debug_aux")
        return xyz, dn

    def debug_quadrature(self, fgrid: torch.Tensor, stream=None) -> torch.Tensor:
        out = torch.empty((n_coeffs(self.N), 2), dtype=torch.float64, device=fgrid.device)
        _check(lib().hamls_debug_quadrature(self.h, _ptr(fgrid), _ptr(out), _stream(stream)),
               "hamls_debug_quadrature")
        return out

    def debug_gl(self, stream=None):
        dev = torch.device("cuda")
        t = torch.empty(self.N + 1, dtype=torch.float64, device=dev)
        w = torch.empty(self.N + 1, dtype=torch.float64, device=dev)
        _check(lib().hamls_debug_gl(self.h, _ptr(t), _ptr(w), _stream(stream)), "hamls_debug_gl")
        return t, w

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().hamls_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cells_noalloc(nodes: torch.Tensor, bands: int, cells: int, keys_sorted: torch.Tensor, perm: torch.Tensor,
                  cell_start: torch.Tensor, stream=None):
    """The cell-list build without device allocation (hamls_cells_noalloc):
    all arguments are caller-owned device tensors (int32 views of uint32)."""
    _check(lib().hamls_cells_noalloc(_ptr(nodes), int(nodes.shape[0]), int(bands), int(cells), _ptr(keys_sorted),
                                     _ptr(perm), _ptr(cell_start), _stream(stream)), "hamls_cells_noalloc")


def plan_footprint(M: int, N: int, K: int, params: Optional[Params] = None, **kw) -> int:
    """Device bytes a plan for (M, N, K) would allocate (hamls_plan_footprint)."""
    p = params if params is not None else default_params(**kw)
    b = ctypes.c_size_t()
    _check(lib().hamls_plan_footprint(int(M), int(N), int(K), ctypes.byref(p), ctypes.byref(b)),
           "hamls_plan_footprint")
    return int(b.value)


def status_from_flags(flags: int) -> int:
    """The hamls_status (0 = ok) for a status word from Plan.status_async."""
    return int(lib().hamls_status_from_flags(int(flags) & 0xFFFFFFFF))


def debug_tc_gemm(A: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
    """C = A B^T on the tensor cores (3xTF32, FP32 accumulation): A (M, K)
    and B (N, K) contiguous float32 device tensors, K a multiple of 4."""
    M, K = A.shape
    N = B.shape[0]
    C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    _check(lib().hamls_debug_tc_gemm(_ptr(A), _ptr(B), _ptr(C), M, N, K, _stream(stream)), "hamls_debug_tc_gemm")
    return C


def to_complex(coeffs: torch.Tensor) -> np.ndarray:
    """(ncoef, 2) float64 -> complex128 numpy (packed m-major)."""
    c = coeffs.detach().cpu().numpy()
    return c[:, 0] + 1j * c[:, 1]
