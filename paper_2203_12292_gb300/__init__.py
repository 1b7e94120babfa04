"""Python binding of libgcmg (global-coarsening matrix-free multigrid on one
GB300).  Argument marshalling only: every step runs in the library's CUDA
kernels; PyTorch provides device memory and the stream.

The library is built in-tree by ``paper_2203_12292_gb300.build.build()``;
importing this module does not build it, and every call fails loudly if the
shared library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgcmg.so")

_c_int, _c_double, _c_void_p, _c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64

PRED_ALL, PRED_OCTANT_CENTRE, PRED_SPHERE, PRED_SHELL, PRED_OCTANT_STRICT = 0, 1, 2, 3, 4

STAGES = ["vmult", "presmooth", "residual", "restrict", "coarse", "prolongate", "postsmooth", "cg_vmult",
          "cg_vector", "learned"]

SMOOTHER_CHEBYSHEV, SMOOTHER_MLP_AUGMENT, SMOOTHER_MLP_REPLACE = 0, 1, 2
FUNC_GAUSSIAN, FUNC_POLYNOMIAL = 2, 3  # manufactured solutions of rhs_dirichlet
GEOM_CARTESIAN, GEOM_WARP = 0, 1  # cell geometry of set_geometry

ERRORS = {1: "GCMG_ERR_ARG", 2: "GCMG_ERR_CUDA", 3: "GCMG_ERR_OOM", 4: "GCMG_ERR_NOT_CONVERGED",
          5: "GCMG_ERR_BREAKDOWN", 6: "GCMG_ERR_INTERNAL"}


class GcmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class RefineStep(ctypes.Structure):
    _fields_ = [("pred", _c_int), ("a", _c_double), ("b", _c_double), ("c", _c_double), ("d", _c_double)]


class Config(ctypes.Structure):
    _fields_ = [("degree", _c_int), ("p_coarsening", _c_int), ("mg_fp32", _c_int), ("cheb_degree", _c_int),
                ("smoothing_range", _c_double), ("eig_steps", _c_int), ("eig_safety", _c_double),
                ("tile_cells", _c_int), ("cell_kernel", _c_int), ("cell_threads", _c_int),
                ("local_smoothing", _c_int), ("transfer_chunk", _c_int)]


class LevelInfo(ctypes.Structure):
    _fields_ = [("n_free", _c_int64), ("n_cells", _c_int64), ("degree", _c_int), ("n_tiles", _c_int),
                ("tile_cells", _c_int), ("max_local", _c_int), ("fp32", _c_int), ("n_halo", _c_int64)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", _c_int), ("r0", _c_double), ("rel_residual", _c_double), ("status", _c_int)]


class PersistentInfo(ctypes.Structure):
    _fields_ = [("grid", _c_int), ("smem_bytes", _c_int), ("ops", ctypes.c_longlong), ("steps", _c_int),
                ("in_graph", _c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("degree", _c_int), ("tile_cells", _c_int), ("cell_kernel", _c_int), ("cell_threads", _c_int),
                ("gdofs", _c_double)]


_SIGS = {
    "gcmg_last_error": (ctypes.c_char_p, []),
    "gcmg_launch_count": (_c_int64, []),
    "gcmg_fma_peak": (_c_int, [_c_int, _c_int, _c_void_p, ctypes.POINTER(_c_double)]),
    "gcmg_mesh_create": (_c_int, [_c_double, _c_double, _c_int, ctypes.POINTER(RefineStep), ctypes.POINTER(_c_void_p)]),
    "gcmg_mesh_destroy": (None, [_c_void_p]),
    "gcmg_mesh_num_levels": (_c_int, [_c_void_p, ctypes.POINTER(_c_int)]),
    "gcmg_mesh_level_cells": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(_c_int64)]),
    "gcmg_mesh_dof_coords": (_c_int, [_c_void_p, _c_int, _c_int, _c_int, ctypes.POINTER(_c_int64), _c_void_p]),
    "gcmg_mesh_check_level": (_c_int, [_c_void_p, _c_int, _c_int, _c_int]),
    "gcmg_config_default": (_c_int, [ctypes.POINTER(Config)]),
    "gcmg_setup": (_c_int, [_c_void_p, ctypes.POINTER(Config), _c_void_p, ctypes.POINTER(_c_void_p)]),
    "gcmg_destroy": (None, [_c_void_p]),
    "gcmg_set_stream": (_c_int, [_c_void_p, _c_void_p]),
    "gcmg_num_levels": (_c_int, [_c_void_p, ctypes.POINTER(_c_int)]),
    "gcmg_get_level_info": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(LevelInfo)]),
    "gcmg_level_dof_coords": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "gcmg_level_edge_dofs": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p]),
    "gcmg_vmult": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p]),
    "gcmg_vmult_host": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p]),
    "gcmg_vmult_host_many": (_c_int, [_c_void_p, _c_int, _c_int, _c_int, ctypes.POINTER(_c_void_p),
                                      ctypes.POINTER(_c_void_p)]),
    "gcmg_dot": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int64, _c_void_p]),
    "gcmg_dot_noalloc": (_c_int, [_c_void_p, _c_void_p, _c_int64, _c_void_p, _c_void_p]),
    "gcmg_set_profiling": (_c_int, [_c_void_p, _c_int]),
    "gcmg_set_graphs": (_c_int, [_c_void_p, _c_int]),
    "gcmg_get_profile": (_c_int, [_c_void_p, _c_int, _c_int, ctypes.POINTER(_c_int64), ctypes.POINTER(_c_double)]),
    "gcmg_diagonal": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "gcmg_rhs": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_double, _c_void_p]),
    "gcmg_rhs_dirichlet": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p]),
    "gcmg_set_coefficient": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "gcmg_set_geometry": (_c_int, [_c_void_p, _c_int, _c_double]),
    "gcmg_get_coefficient": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "gcmg_quadrature_points": (_c_int, [_c_void_p, _c_void_p]),
    "gcmg_get_lambda": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(_c_double)]),
    "gcmg_set_lambda": (_c_int, [_c_void_p, _c_int, _c_double]),
    "gcmg_smooth": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_int]),
    "gcmg_prolongate_add": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p]),
    "gcmg_restrict_add": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p]),
    "gcmg_coarse_solve": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p]),
    "gcmg_vcycle": (_c_int, [_c_void_p, _c_void_p, _c_void_p]),
    "gcmg_vcycle_cgc": (_c_int, [_c_void_p, _c_void_p, _c_void_p]),
    "gcmg_residual": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p, _c_void_p, _c_void_p]),
    "gcmg_cg_solve": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_double, _c_int, ctypes.POINTER(SolveStats)]),
    "gcmg_mlp_create": (_c_int, [_c_int, _c_int, _c_int, ctypes.POINTER(_c_void_p)]),
    "gcmg_mlp_destroy": (None, [_c_void_p]),
    "gcmg_mlp_num_params": (_c_int, [_c_void_p, ctypes.POINTER(_c_int64)]),
    "gcmg_mlp_set_params": (_c_int, [_c_void_p, _c_void_p, _c_void_p]),
    "gcmg_mlp_get_params": (_c_int, [_c_void_p, _c_void_p, _c_void_p]),
    "gcmg_mlp_forward": (_c_int, [_c_void_p, _c_void_p, _c_int64, _c_void_p, _c_void_p]),
    "gcmg_mlp_gradient": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_int64, _c_void_p, _c_void_p,
                                   _c_void_p]),
    "gcmg_mlp_train": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_int64, _c_void_p, _c_int64, _c_int,
                                ctypes.c_float, _c_void_p, _c_void_p]),
    "gcmg_level_cells": (_c_int, [_c_void_p, _c_int, _c_void_p]),
    "gcmg_cell_gather": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_int64, _c_void_p, _c_void_p]),
    "gcmg_mlp_samples": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_void_p, _c_void_p, _c_int64, _c_void_p,
                                  _c_void_p, _c_void_p, _c_void_p]),
    "gcmg_mlp_correct": (_c_int, [_c_void_p, _c_int, _c_void_p, _c_int, _c_void_p, _c_void_p]),
    "gcmg_set_smoother": (_c_int, [_c_void_p, _c_int, _c_int, _c_void_p]),
    "gcmg_wait_timeouts": (_c_int, [ctypes.POINTER(ctypes.c_uint), _c_int]),
    "gcmg_point_values": (_c_int, [_c_void_p, _c_int64, ctypes.c_uint64, _c_void_p]),
    "gcmg_autotune": (_c_int, [_c_void_p, _c_int, _c_int, _c_int, _c_void_p, ctypes.POINTER(Tuning),
                               ctypes.POINTER(Tuning), ctypes.POINTER(_c_int)]),
    "gcmg_batch_create": (_c_int, [_c_int, ctypes.POINTER(_c_void_p), ctypes.POINTER(Config), _c_int, _c_void_p,
                                   ctypes.POINTER(_c_void_p)]),
    "gcmg_batch_destroy": (None, [_c_void_p]),
    "gcmg_batch_size": (_c_int, [_c_void_p, ctypes.POINTER(_c_int)]),
    "gcmg_batch_handle": (_c_int, [_c_void_p, _c_int, ctypes.POINTER(_c_void_p)]),
    "gcmg_batch_cg_solve": (_c_int, [_c_void_p, ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p), _c_double,
                                     _c_int, ctypes.POINTER(SolveStats)]),
    "gcmg_batch_cg_solve_persistent": (_c_int, [_c_void_p, ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p),
                                                _c_double, _c_int, ctypes.POINTER(SolveStats)]),
    "gcmg_batch_persistent_info": (_c_int, [_c_void_p, ctypes.POINTER(PersistentInfo)]),
    "gcmg_batch_persistent_wait_test": (_c_int, [_c_void_p, _c_int, ctypes.c_uint]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libgcmg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2203_12292_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernel launches issued by libgcmg so far."""
    return int(lib().gcmg_launch_count())


def fma_peak(fp64: bool, iters: int = 1 << 16) -> float:
    """Measured peak of the CUDA cores of the current device in TFLOP/s
    (fp32, or native fp64), on the current torch stream."""
    import torch
    out = _c_double()
    _check(lib().gcmg_fma_peak(int(fp64), iters, _c_void_p(torch.cuda.current_stream().cuda_stream),
                               ctypes.byref(out)))
    return out.value


def wait_timeouts(reset: bool = False) -> int:
    """Bounded tensor-core waits that gave up since the library was loaded
    (or the last reset); synchronises the device."""
    out = ctypes.c_uint()
    _check(lib().gcmg_wait_timeouts(ctypes.byref(out), int(reset)))
    return out.value


def exported_symbols() -> Sequence[str]:
    return list(_SIGS)


def _check(rc: int) -> None:
    if rc != 0:
        raise GcmgError(rc, lib().gcmg_last_error().decode())


def _steps(steps: Sequence[Tuple]) -> ctypes.Array:
    arr = (RefineStep * max(len(steps), 1))()
    for i, s in enumerate(steps):
        vals = list(s) + [0.0] * (5 - len(s))
        arr[i] = RefineStep(int(vals[0]), *[float(v) for v in vals[1:5]])
    return arr


class Mesh:
    """Octree mesh and its global-coarsening hierarchy (host only).

    ``steps`` is a sequence of (pred, a, b[, c, d]) refinement steps."""

    def __init__(self, lo: float, hi: float, steps: Sequence[Tuple]):
        p = _c_void_p()
        arr = _steps(steps)
        _check(lib().gcmg_mesh_create(lo, hi, len(steps), arr, ctypes.byref(p)))
        self._p = p

    @classmethod
    def from_recipe(cls, recipe) -> "Mesh":
        return cls(recipe.lo, recipe.hi, [(s.pred, s.a, s.b, s.c, s.d) for s in recipe.steps])

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.gcmg_mesh_destroy(self._p)
            self._p = None

    @property
    def num_levels(self) -> int:
        n = _c_int()
        _check(lib().gcmg_mesh_num_levels(self._p, ctypes.byref(n)))
        return n.value

    def level_cells(self, level: int) -> int:
        n = _c_int64()
        _check(lib().gcmg_mesh_level_cells(self._p, level, ctypes.byref(n)))
        return n.value

    def check_level(self, level: int, degree: int, tile_cells: int = 0) -> None:
        """Validate the tile data of a level on the host (raises GcmgError)."""
        _check(lib().gcmg_mesh_check_level(self._p, level, degree, tile_cells))

    def dof_coords(self, level: int, degree: int, tile_cells: int = 0) -> np.ndarray:
        n = _c_int64()
        _check(lib().gcmg_mesh_dof_coords(self._p, level, degree, tile_cells, ctypes.byref(n), None))
        xyz = np.empty((n.value, 3), dtype=np.float64)
        _check(lib().gcmg_mesh_dof_coords(self._p, level, degree, tile_cells, ctypes.byref(n),
                                          xyz.ctypes.data_as(_c_void_p)))
        return xyz


def _ptr(t, n: Optional[int] = None, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} entries, got {t.numel()}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return _c_void_p(t.data_ptr() if t.numel() else None)


def _is64(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return 1
    if t.dtype == torch.float32:
        return 0
    raise ValueError("vectors must be float32 or float64")


def make_config(degree: int, p_coarsening: bool = False, mg_fp32: bool = True, tile_cells: int = 0,
                cheb_degree: int = 3, smoothing_range: float = 20.0, eig_steps: int = 12, eig_safety: float = 1.2,
                cell_kernel: int = 0, cell_threads: int = 0, local_smoothing: bool = False,
                transfer_chunk: int = 0) -> Config:
    cfg = Config()
    _check(lib().gcmg_config_default(ctypes.byref(cfg)))
    cfg.degree, cfg.p_coarsening, cfg.mg_fp32 = degree, int(p_coarsening), int(mg_fp32)
    cfg.tile_cells, cfg.cheb_degree, cfg.smoothing_range = tile_cells, cheb_degree, smoothing_range
    cfg.eig_steps, cfg.eig_safety, cfg.cell_kernel = eig_steps, eig_safety, cell_kernel
    cfg.cell_threads = cell_threads
    cfg.local_smoothing = int(local_smoothing)
    cfg.transfer_chunk = transfer_chunk
    return cfg


class Multigrid:
    """All levels of one problem on the current CUDA device, set up on the
    current torch stream."""

    def __init__(self, mesh: Mesh, degree: int, p_coarsening: bool = False, mg_fp32: bool = True,
                 tile_cells: int = 0, cheb_degree: int = 3, smoothing_range: float = 20.0,
                 eig_steps: int = 12, eig_safety: float = 1.2, cell_kernel: int = 0, cell_threads: int = 0,
                 local_smoothing: bool = False, transfer_chunk: int = 0, _handle=None, _owner=None):
        import torch
        self.mesh = mesh
        self.stream = torch.cuda.current_stream()
        if _handle is not None:  # a handle owned by a Batch
            self._h, self._owned, self._owner = _handle, False, _owner
        else:
            cfg = make_config(degree, p_coarsening, mg_fp32, tile_cells, cheb_degree, smoothing_range, eig_steps,
                              eig_safety, cell_kernel, cell_threads, local_smoothing, transfer_chunk)
            h = _c_void_p()
            _check(lib().gcmg_setup(mesh._p, ctypes.byref(cfg), _c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
            self._h, self._owned = h, True
        self.num_levels = self._num_levels()
        self.info = [self.level_info(l) for l in range(self.num_levels)]
        # local smoothing: levels 0 .. num_levels - 2 are the refinement levels, the last one the active mesh
        self.local_smoothing = bool(local_smoothing) and _handle is None

    def __del__(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", False) and _lib is not None:
            _lib.gcmg_destroy(self._h)
        self._h = None

    def _num_levels(self) -> int:
        n = _c_int()
        _check(lib().gcmg_num_levels(self._h, ctypes.byref(n)))
        return n.value

    def level_info(self, level: int) -> LevelInfo:
        info = LevelInfo()
        _check(lib().gcmg_get_level_info(self._h, level, ctypes.byref(info)))
        return info

    def n_free(self, level: int = -1) -> int:
        return self.info[level].n_free

    @property
    def finest(self) -> int:
        return self.num_levels - 1

    def edge_dofs(self, level: int) -> np.ndarray:
        """local smoothing: indices of the refinement-edge DoFs of a level"""
        n = _c_int64()
        _check(lib().gcmg_level_edge_dofs(self._h, level, ctypes.byref(n), None))
        out = np.empty(n.value, dtype=np.int32)
        if n.value:
            _check(lib().gcmg_level_edge_dofs(self._h, level, ctypes.byref(n), out.ctypes.data_as(_c_void_p)))
        return out

    def dof_coords(self, level: int) -> np.ndarray:
        xyz = np.empty((self.n_free(level), 3), dtype=np.float64)
        _check(lib().gcmg_level_dof_coords(self._h, level, xyz.ctypes.data_as(_c_void_p)))
        return xyz

    def set_stream(self, stream) -> None:
        self.stream = stream
        _check(lib().gcmg_set_stream(self._h, _c_void_p(stream.cuda_stream)))

    def vmult(self, level: int, src, dst) -> None:
        n = self.n_free(level)
        _check(lib().gcmg_vmult(self._h, level, _is64(src), _ptr(src, n, src.dtype), _ptr(dst, n, src.dtype)))

    def vmult_host(self, level: int, src: np.ndarray, dst: np.ndarray) -> None:
        """Operator with host (numpy) vectors; copies in and out, synchronous."""
        n = self.n_free(level)
        if src.dtype not in (np.float32, np.float64) or dst.dtype != src.dtype or len(src) != n or len(dst) != n:
            raise ValueError("host vectors must be float32/float64 of length n_free")
        if not (src.flags.c_contiguous and dst.flags.c_contiguous):
            raise ValueError("host vectors must be contiguous")
        _check(lib().gcmg_vmult_host(self._h, level, int(src.dtype == np.float64), src.ctypes.data_as(_c_void_p),
                                     dst.ctypes.data_as(_c_void_p)))

    def vmult_host_many(self, level: int, srcs: Sequence[np.ndarray], dsts: Sequence[np.ndarray]) -> None:
        """Operator on several host (numpy) vectors, the copies of neighbouring
        vectors overlapped with the operators; synchronous."""
        n = self.n_free(level)
        if len(srcs) != len(dsts):
            raise ValueError("as many outputs as inputs")
        for a, b in zip(srcs, dsts):
            if a.dtype not in (np.float32, np.float64) or b.dtype != a.dtype or a.dtype != srcs[0].dtype:
                raise ValueError("host vectors must all be float32 or all float64")
            if len(a) != n or len(b) != n or not (a.flags.c_contiguous and b.flags.c_contiguous):
                raise ValueError("host vectors must be contiguous with n_free values")
        k = len(srcs)
        sarr = (_c_void_p * max(k, 1))(*[a.ctypes.data_as(_c_void_p) for a in srcs])
        darr = (_c_void_p * max(k, 1))(*[b.ctypes.data_as(_c_void_p) for b in dsts])
        f64 = int(k > 0 and srcs[0].dtype == np.float64)
        _check(lib().gcmg_vmult_host_many(self._h, level, f64, k, sarr, darr))

    def dot(self, x, y, out=None):
        """fp64 inner product on the device (deterministic); returns a 1-element tensor."""
        import torch
        n = x.numel()
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(lib().gcmg_dot(self._h, _ptr(x, n, torch.float64), _ptr(y, n, torch.float64), n, _ptr(out, 1)))
        return out

    def set_graphs(self, on: bool) -> None:
        """Run the V-cycle and CG operator steps as captured CUDA graphs (default) or eagerly."""
        _check(lib().gcmg_set_graphs(self._h, int(on)))

    def set_profiling(self, on: bool) -> None:
        _check(lib().gcmg_set_profiling(self._h, int(on)))

    def profile(self, level: int, stage: str):
        """(launch count, milliseconds) accumulated for a level and stage."""
        c, ms = _c_int64(), _c_double()
        _check(lib().gcmg_get_profile(self._h, level, STAGES.index(stage), ctypes.byref(c), ctypes.byref(ms)))
        return c.value, ms.value

    def diagonal(self, level: int):
        import torch
        d = torch.empty(self.n_free(level), dtype=torch.float64, device="cuda")
        _check(lib().gcmg_diagonal(self._h, level, _ptr(d)))
        return d

    def rhs(self, fourier=None):
        """b = C^T F on the finest level; ``fourier`` = (kappa (m,3), phi (m,), amp) or None for f = 1."""
        import torch
        b = torch.empty(self.n_free(self.finest), dtype=torch.float64, device="cuda")
        if fourier is None:
            _check(lib().gcmg_rhs(self._h, 0, None, 1.0, _ptr(b)))
        else:
            kappa, phi, amp = fourier
            modes = np.ascontiguousarray(np.concatenate([np.asarray(kappa, np.float64),
                                                         np.asarray(phi, np.float64)[:, None]], axis=1))
            _check(lib().gcmg_rhs(self._h, len(phi), modes.ctypes.data_as(_c_void_p), float(amp), _ptr(b)))
        return b

    def rhs_dirichlet(self, kind: int, params):
        """b = C^T (F - A_all u_g) for the manufactured solution u (Dirichlet
        data u, f = -Lap u): kind FUNC_GAUSSIAN with params (alpha, x0, y0, z0),
        or FUNC_POLYNOMIAL with params = terms (c, a, b, e)."""
        import torch
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1, 4))
        b = torch.empty(self.n_free(self.finest), dtype=torch.float64, device="cuda")
        _check(lib().gcmg_rhs_dirichlet(self._h, int(kind), len(p), p.ctypes.data_as(_c_void_p), _ptr(b)))
        return b

    def quadrature_points(self):
        """Gauss points of every finest cell, (n_cells, (k+1)^3, 3) on the device."""
        import torch
        n3 = (self.info[self.finest].degree + 1) ** 3
        xyz = torch.empty((self.n_cells(self.finest), n3, 3), dtype=torch.float64, device="cuda")
        _check(lib().gcmg_quadrature_points(self._h, _ptr(xyz)))
        return xyz

    def set_coefficient(self, nu) -> None:
        """nu: device fp64, per finest cell (n_cells,) or per Gauss point
        (n_cells, (k+1)^3); see gcmg_set_coefficient."""
        import torch
        nc = self.n_cells(self.finest)
        assert nu.dtype == torch.float64 and nu.is_cuda and nu.is_contiguous()
        assert nu.numel() % max(nc, 1) == 0
        per = nu.numel() // nc if nc else 1
        _check(lib().gcmg_set_coefficient(self._h, per, _ptr(nu)))

    def set_geometry(self, kind: int, eps: float = 0.0) -> None:
        """GEOM_WARP: the cells mapped by Phi(x) = x + eps (x1 x2, 2 x2 x0, x0 x1 / 2);
        GEOM_CARTESIAN: back to Cartesian cells (see gcmg_set_geometry)."""
        _check(lib().gcmg_set_geometry(self._h, int(kind), float(eps)))

    def get_coefficient(self, level: int):
        import torch
        nu = torch.empty(self.n_cells(level), dtype=torch.float64, device="cuda")
        _check(lib().gcmg_get_coefficient(self._h, level, _ptr(nu)))
        return nu

    def get_lambda(self, level: int) -> float:
        v = _c_double()
        _check(lib().gcmg_get_lambda(self._h, level, ctypes.byref(v)))
        return v.value

    def set_lambda(self, level: int, lam: float) -> None:
        _check(lib().gcmg_set_lambda(self._h, level, lam))

    def smooth(self, level: int, x, b, zero_init: bool) -> None:
        n = self.n_free(level)
        _check(lib().gcmg_smooth(self._h, level, _is64(x), _ptr(x, n, x.dtype), _ptr(b, n, x.dtype), int(zero_init)))

    def prolongate_add(self, fine_level: int, coarse, fine) -> None:
        _check(lib().gcmg_prolongate_add(self._h, fine_level, _is64(fine), _ptr(coarse, self.n_free(fine_level - 1), fine.dtype),
                                         _ptr(fine, self.n_free(fine_level), fine.dtype)))

    def restrict_add(self, fine_level: int, fine, coarse) -> None:
        _check(lib().gcmg_restrict_add(self._h, fine_level, _is64(fine), _ptr(fine, self.n_free(fine_level), fine.dtype),
                                       _ptr(coarse, self.n_free(fine_level - 1), fine.dtype)))

    def coarse_solve(self, b, x) -> None:
        n = self.n_free(0)
        _check(lib().gcmg_coarse_solve(self._h, _is64(b), _ptr(b, n, b.dtype), _ptr(x, n, b.dtype)))

    def vcycle(self, b, x) -> None:
        import torch
        n = self.n_free(self.finest)
        _check(lib().gcmg_vcycle(self._h, _ptr(b, n, torch.float64), _ptr(x, n, torch.float64)))

    def vcycle_cgc(self, b, x) -> None:
        """V-cycle stopped after the finest-level prolongation (coarse-grid corrected iterate)."""
        import torch
        n = self.n_free(self.finest)
        _check(lib().gcmg_vcycle_cgc(self._h, _ptr(b, n, torch.float64), _ptr(x, n, torch.float64)))

    def residual(self, level: int, b, x, r) -> None:
        """r = b - A x on a level."""
        n = self.n_free(level)
        _check(lib().gcmg_residual(self._h, level, _is64(x), _ptr(b, n, x.dtype), _ptr(x, n, x.dtype),
                                   _ptr(r, n, x.dtype)))

    def cg_solve(self, b, x, rtol: float = 1e-8, maxit: int = 100, raise_on_fail: bool = True) -> SolveStats:
        import torch
        n = self.n_free(self.finest)
        st = SolveStats()
        rc = lib().gcmg_cg_solve(self._h, _ptr(b, n, torch.float64), _ptr(x, n, torch.float64), rtol, maxit,
                                 ctypes.byref(st))
        if rc != 0 and (raise_on_fail or rc not in (4, 5)):
            _check(rc)
        return st

    # ---- learned smoother --------------------------------------------------
    def n_cells(self, level: int) -> int:
        return self.info[level].n_cells

    def _check_cells(self, level: int, cells) -> None:
        if cells.numel() and (int(cells.min()) < 0 or int(cells.max()) >= self.n_cells(level)):
            raise ValueError("cell index out of range")

    def level_cells(self, level: int) -> np.ndarray:
        """(l, i, j, k) of every cell in the library's cell order."""
        out = np.empty((self.n_cells(level), 4), dtype=np.int32)
        _check(lib().gcmg_level_cells(self._h, level, out.ctypes.data_as(_c_void_p)))
        return out

    def cell_gather(self, level: int, x, cells=None):
        """Values of the fp64 vector x at the support points of the cells
        (all cells when ``cells`` is None): (n_cells, (k+1)^3) fp64 tensor."""
        import torch
        n3 = (self.info[level].degree + 1) ** 3
        nc = self.n_cells(level) if cells is None else cells.numel()
        if cells is not None:
            self._check_cells(level, cells)
        out = torch.empty((nc, n3), dtype=torch.float64, device="cuda")
        cp = None if cells is None else _ptr(cells, nc, torch.int32)
        _check(lib().gcmg_cell_gather(self._h, level, _ptr(x, self.n_free(level), torch.float64), nc, cp,
                                      _ptr(out)))
        return out

    def mlp_samples(self, level: int, b, x, xstar, cells):
        """Training rows (X, T, W) of the cells from the residual b - A x and
        the error xstar - x (fp64 vectors; xstar None gives T = None)."""
        import torch
        self._check_cells(level, cells)
        n3 = (self.info[level].degree + 1) ** 3
        nc = cells.numel()
        X = torch.empty((nc, 2 * n3), dtype=torch.float32, device="cuda")
        T = torch.empty((nc, n3), dtype=torch.float32, device="cuda") if xstar is not None else None
        W = torch.empty(nc, dtype=torch.float32, device="cuda")
        n = self.n_free(level)
        _check(lib().gcmg_mlp_samples(self._h, level, _ptr(b, n, torch.float64), _ptr(x, n, torch.float64),
                                      None if xstar is None else _ptr(xstar, n, torch.float64), nc,
                                      _ptr(cells, nc, torch.int32), _ptr(X), None if T is None else _ptr(T),
                                      _ptr(W)))
        return X, T, W

    def mlp_correct(self, level: int, net: "MLP", r, x) -> None:
        """x += the learned correction of ``net`` for the residual r."""
        n = self.n_free(level)
        _check(lib().gcmg_mlp_correct(self._h, level, net._p, _is64(x), _ptr(r, n, x.dtype), _ptr(x, n, x.dtype)))

    def set_smoother(self, level: int, kind: int, net: "Optional[MLP]" = None) -> None:
        _check(lib().gcmg_set_smoother(self._h, level, kind, None if net is None else net._p))


class MLP:
    """Per-cell network of the learned smoother (device parameters, Adam state)."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int):
        p = _c_void_p()
        _check(lib().gcmg_mlp_create(n_in, n_hidden, n_out, ctypes.byref(p)))
        self._p = p
        self.shape = (n_in, n_hidden, n_out)

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.gcmg_mlp_destroy(self._p)
            self._p = None

    @property
    def num_params(self) -> int:
        n = _c_int64()
        _check(lib().gcmg_mlp_num_params(self._p, ctypes.byref(n)))
        return n.value

    def _stream(self):
        import torch
        return _c_void_p(torch.cuda.current_stream().cuda_stream)

    def set_params(self, theta) -> None:
        import torch
        _check(lib().gcmg_mlp_set_params(self._p, _ptr(theta, self.num_params, torch.float32), self._stream()))

    def get_params(self):
        import torch
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _check(lib().gcmg_mlp_get_params(self._p, _ptr(out), self._stream()))
        return out

    def forward(self, X):
        import torch
        n = X.shape[0]
        Y = torch.empty((n, self.shape[2]), dtype=torch.float32, device="cuda")
        _check(lib().gcmg_mlp_forward(self._p, _ptr(X, n * self.shape[0], torch.float32), n, _ptr(Y),
                                      self._stream()))
        return Y

    def gradient(self, X, T, W=None):
        """(loss tensor (1,), gradient tensor (num_params,)); W: row weights or None."""
        import torch
        n = X.shape[0]
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        L = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(lib().gcmg_mlp_gradient(self._p, _ptr(X, n * self.shape[0], torch.float32),
                                       _ptr(T, n * self.shape[2], torch.float32),
                                       None if W is None else _ptr(W, n, torch.float32), n, _ptr(g), _ptr(L),
                                       self._stream()))
        return L, g

    def train(self, X, T, order, batch: int, lr: float = 1e-3, W=None):
        """Adam over consecutive batches of ``order``; returns the per-step losses."""
        import torch
        n = X.shape[0]
        if order.numel() and (int(order.min()) < 0 or int(order.max()) >= n):
            raise ValueError("sample order out of range")
        steps = order.numel() // batch
        losses = torch.empty(max(steps, 1), dtype=torch.float32, device="cuda")
        _check(lib().gcmg_mlp_train(self._p, _ptr(X, n * self.shape[0], torch.float32),
                                    _ptr(T, n * self.shape[2], torch.float32),
                                    None if W is None else _ptr(W, n, torch.float32), n,
                                    _ptr(order, order.numel(), torch.int32), order.numel(), batch, float(lr),
                                    _ptr(losses), self._stream()))
        return losses[:steps]


def point_values(xyz: np.ndarray, seed: int) -> np.ndarray:
    """Position-keyed uniform values in [-1, 1) computed by the library."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.empty(len(xyz), dtype=np.float64)
    _check(lib().gcmg_point_values(xyz.ctypes.data_as(_c_void_p), len(xyz), seed, out.ctypes.data_as(_c_void_p)))
    return out


def autotune(probe: Mesh, degree: int, mg_fp32: bool = True, reps: int = 20):
    """(best, all candidates) of the operator autotuner for one degree."""
    import torch
    best = Tuning()
    allc = (Tuning * 16)()  # GCMG_AUTOTUNE_MAX
    n = _c_int()
    _check(lib().gcmg_autotune(probe._p, degree, int(mg_fp32), reps, _c_void_p(torch.cuda.current_stream().cuda_stream),
                               ctypes.byref(best), allc, ctypes.byref(n)))
    return best, [allc[i] for i in range(n.value)]


class Batch:
    """Independent problems set up together and solved by one graph launch."""

    def __init__(self, meshes: Sequence[Mesh], configs: Sequence[Config], n_threads: int = 0):
        import torch
        n = len(meshes)
        arr = (_c_void_p * n)(*[m._p for m in meshes])
        cfgs = (Config * n)(*configs)
        self.stream = torch.cuda.current_stream()
        p = _c_void_p()
        _check(lib().gcmg_batch_create(n, arr, cfgs, n_threads, _c_void_p(self.stream.cuda_stream), ctypes.byref(p)))
        self._p = p
        self.meshes = list(meshes)
        self.problems = []
        for i in range(n):
            h = _c_void_p()
            _check(lib().gcmg_batch_handle(p, i, ctypes.byref(h)))
            self.problems.append(Multigrid(meshes[i], configs[i].degree, _handle=h, _owner=self))

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            for m in getattr(self, "problems", []):
                m._h = None
            _lib.gcmg_batch_destroy(self._p)
            self._p = None

    def __len__(self) -> int:
        return len(self.problems)

    def cg_solve(self, bs, xs, rtol: float = 1e-8, maxit: int = 100, persistent: bool = False):
        """CG to rtol for every problem in one graph launch (persistent: the
        whole batch in one persistent kernel); returns the per-problem stats."""
        import torch
        n = len(self.problems)
        assert len(bs) == n and len(xs) == n
        for m, b, x in zip(self.problems, bs, xs):
            nf = m.n_free(m.finest)
            _ptr(b, nf, torch.float64)
            _ptr(x, nf, torch.float64)
        barr = (_c_void_p * n)(*[b.data_ptr() if b.numel() else None for b in bs])
        xarr = (_c_void_p * n)(*[x.data_ptr() if x.numel() else None for x in xs])
        st = (SolveStats * n)()
        fn = lib().gcmg_batch_cg_solve_persistent if persistent else lib().gcmg_batch_cg_solve
        _check(fn(self._p, barr, xarr, rtol, maxit, st))
        return [st[i] for i in range(n)]

    def persistent_wait_test(self, absent_cta: int = -1, spin_limit: int = 1 << 25) -> None:
        """Test of the persistent kernel's bounded waits: CTA absent_cta leaves
        before the first grid barrier; (-1, 1 << 25) restores the normal launch."""
        _check(lib().gcmg_batch_persistent_wait_test(self._p, absent_cta, spin_limit))

    def persistent_info(self) -> PersistentInfo:
        """grid, shared memory, operations and steps of the last persistent solve"""
        out = PersistentInfo()
        _check(lib().gcmg_batch_persistent_info(self._p, ctypes.byref(out)))
        return out
