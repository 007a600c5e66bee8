"""GB300 level-set mesher: Python binding of liblsm (the C ABI in include/lsm.h).

This module only marshals arguments: every step of the evaluation and of the
Newton chart solve runs in the library's CUDA kernels.  Arrays may be numpy
arrays (host memory) or torch tensors (host or CUDA); outputs are allocated
on the same side as the input points unless given.  There is no CPU fallback:
without the compiled library or a CUDA device the calls raise.

Names follow the paper (Vico, Greengard, O'Neil, Rachh, arXiv 1909.13356):
Phi, grad Phi (Sec. 4), chart nodes, h, pseudonormals H (Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = ["FP64", "MIXED", "FF", "Context", "Mesh", "Batch", "SolveStats", "LsmError", "lib", "load"]

FP64 = 0
MIXED = 1
FF = 2

NODE_CONVERGED = 0
NODE_MAXITER = 1
NODE_ZERODERIV = 2
NODE_NONFINITE = 3
NODE_CLAMPED_BIT = 256

_ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "MESH", -5: "NOT_CONVERGED", -6: "TIMEOUT",
           -7: "CANCELLED"}

# every symbol include/lsm.h declares
EXPORTS = ("lsm_create", "lsm_destroy", "lsm_last_error", "lsm_launch_count", "lsm_set_profiling",
           "lsm_read_stats", "lsm_mesh_upload", "lsm_mesh_free", "lsm_mesh_get_info", "lsm_eval_phi_grad",
           "lsm_eval_phi_grad_noalloc", "lsm_solve_charts", "lsm_batch_create", "lsm_batch_free",
           "lsm_batch_solve_charts", "lsm_server_create", "lsm_server_submit", "lsm_server_poll", "lsm_server_release",
           "lsm_server_info", "lsm_server_destroy", "lsm_autotune", "lsm_chart_frames", "lsm_gauss_flux",
           "lsm_mesh_upload_sigmax", "lsm_mesh_get_sigma0", "lsm_eval_sigma", "lsm_eval_hessian",
           "lsm_chart_curvature", "lsm_refined_nodes", "lsm_solve_charts_nodes", "lsm_chart_frames_nodes",
           "lsm_gauss_flux_nodes", "lsm_check_error", "lsm_test_inject_wait_timeout", "lsm_measure_peaks",
           "lsm_server_cancel", "lsm_batch_autotune",
           "lsm_mesh_upload_quadratic", "lsm_flux_per_triangle", "lsm_refine_adaptive")


class LsmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lsm error {code} ({_ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Quad(ctypes.Structure):
    _fields_ = [("n_gl", ctypes.c_int32), ("subdiv", ctypes.c_int32)]


class _Options(ctypes.Structure):
    _fields_ = [("cutoff_fp64", ctypes.c_double), ("cutoff_mixed", ctypes.c_double),
                ("mixed_switch", ctypes.c_double), ("mixed_accept", ctypes.c_double),
                ("tree_degree", ctypes.c_int32), ("tree_theta", ctypes.c_float),
                ("tree_min_sources", ctypes.c_int32), ("tree_ff_degree", ctypes.c_int32),
                ("tree_ff_theta", ctypes.c_float), ("tree_ff_min_sources", ctypes.c_int32),
                ("tree_grid", ctypes.c_int32), ("tree_ff_cluster", ctypes.c_int32), ("tree_cluster", ctypes.c_int32),
                ("ff_block", ctypes.c_int32), ("mixed_block", ctypes.c_int32),
                ("newton_tree_degree", ctypes.c_int32), ("newton_tree_theta", ctypes.c_float),
                ("newton_cutoff", ctypes.c_float)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("n_converged", ctypes.c_int32), ("n_failed", ctypes.c_int32),
                ("eps_newton", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("evals_fp32", ctypes.c_int64), ("evals_fp64", ctypes.c_int64),
                ("active_per_iter", ctypes.c_int32 * 32), ("evals_near_only", ctypes.c_int64)]


class _CtxStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("pairs_near", ctypes.c_int64),
                ("pairs_far", ctypes.c_int64), ("pair_kernel_launches", ctypes.c_int64),
                ("pair_kernel_ms", ctypes.c_double), ("kind_pairs_near", ctypes.c_int64 * 4),
                ("kind_pairs_far", ctypes.c_int64 * 4), ("kind_launches", ctypes.c_int64 * 4),
                ("kind_ms", ctypes.c_double * 4)]


class _Info(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_sources", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("sigma_min", ctypes.c_double),
                ("sigma_max", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("nv", ctypes.c_int64), ("tris", ctypes.c_void_p),
                ("nt", ctypes.c_int64), ("sigma", ctypes.c_void_p), ("rule", _Quad), ("order", ctypes.c_int32),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("stats", _Stats), ("x", ctypes.POINTER(ctypes.c_double)), ("h", ctypes.POINTER(ctypes.c_double)),
                ("node_status", ctypes.POINTER(ctypes.c_int32)), ("error", ctypes.c_char_p)]


class _Peaks(ctypes.Structure):
    _fields_ = [("ffma_tflops", ctypes.c_double), ("ffma2_tflops", ctypes.c_double),
                ("dfma_tflops", ctypes.c_double), ("rsqrt_gops", ctypes.c_double), ("ex2_gops", ctypes.c_double),
                ("ms", ctypes.c_double * 5)]


class _TuneResult(ctypes.Structure):
    _fields_ = [("use_tree", ctypes.c_int32), ("tree_degree", ctypes.c_int32), ("tree_theta", ctypes.c_float),
                ("candidates", ctypes.c_int32), ("sample_targets", ctypes.c_int64), ("err_phi", ctypes.c_double),
                ("ms_sample", ctypes.c_double), ("ms_direct", ctypes.c_double), ("err_direct", ctypes.c_double),
                ("cutoff", ctypes.c_double), ("targets_per_block", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("max_running", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("in_use_bytes", ctypes.c_int64),
                ("peak_in_use_bytes", ctypes.c_int64), ("now_ms", ctypes.c_double)]


@dataclass
class SolveStats:
    iterations: int
    n_nodes: int
    n_converged: int
    n_failed: int
    eps_newton: float
    max_residual: float
    evals_fp32: int
    evals_fp64: int
    active_per_iter: list
    evals_near_only: int = 0


_lock = threading.Lock()
_lib = None


def load(build_if_needed: bool = True):
    """Load liblsm.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"liblsm.so not built ({_build.LIB}); run paper_1909_13356_gb300/build.py")
        L = ctypes.CDLL(_build.LIB)
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.lsm_create.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(_Options)]
        L.lsm_destroy.argtypes = [P]
        L.lsm_last_error.argtypes = [P]
        L.lsm_last_error.restype = ctypes.c_char_p
        L.lsm_launch_count.argtypes = [P]
        L.lsm_launch_count.restype = I64
        L.lsm_set_profiling.argtypes = [P, I32]
        L.lsm_read_stats.argtypes = [P, ctypes.POINTER(_CtxStats), I32]
        L.lsm_mesh_upload.argtypes = [P, P, I64, P, I64, P, ctypes.POINTER(_Quad), P, ctypes.POINTER(P)]
        L.lsm_mesh_free.argtypes = [P]
        L.lsm_mesh_get_info.argtypes = [P, ctypes.POINTER(_Info)]
        L.lsm_eval_phi_grad.argtypes = [P, P, I64, P, P, I32, P]
        L.lsm_eval_phi_grad_noalloc.argtypes = [P, P, I64, P, P, I32, P]
        L.lsm_solve_charts.argtypes = [P, I32, D, I32, I32, P, P, P, ctypes.POINTER(_Stats), P]
        L.lsm_server_create.argtypes = [P, I32, I64, ctypes.POINTER(P)]
        L.lsm_server_submit.argtypes = [P, ctypes.POINTER(_Request), ctypes.POINTER(I64)]
        L.lsm_server_poll.argtypes = [P, I64, I32, ctypes.POINTER(_Result)]
        L.lsm_server_release.argtypes = [P, I64]
        L.lsm_server_cancel.argtypes = [P, I64]
        L.lsm_server_info.argtypes = [P, ctypes.POINTER(_ServerInfo)]
        L.lsm_server_destroy.argtypes = [P]
        L.lsm_batch_create.argtypes = [P, ctypes.POINTER(P), I32, P, ctypes.POINTER(P)]
        L.lsm_batch_free.argtypes = [P]
        L.lsm_batch_solve_charts.argtypes = [P, I32, D, I32, I32, I32, P, P, P, ctypes.POINTER(_Stats), P]
        L.lsm_autotune.argtypes = [P, P, I64, D, ctypes.POINTER(_TuneResult), P]
        L.lsm_batch_autotune.argtypes = [P, I32, D, ctypes.POINTER(_TuneResult), P]
        L.lsm_chart_frames.argtypes = [P, I32, P, P, P, P, P, P]
        L.lsm_mesh_upload_quadratic.argtypes = [P, P, I64, P, I64, P, ctypes.POINTER(_Quad), P, ctypes.POINTER(P)]
        L.lsm_mesh_upload_sigmax.argtypes = [P, P, I64, P, I64, D, D, ctypes.POINTER(_Quad), P, ctypes.POINTER(P)]
        L.lsm_mesh_get_sigma0.argtypes = [P, ctypes.POINTER(D)]
        L.lsm_eval_sigma.argtypes = [P, P, I64, P, P, P]
        L.lsm_eval_hessian.argtypes = [P, P, I64, P, P]
        L.lsm_chart_curvature.argtypes = [P, I32, P, P, P, P, P, P, P, P, P]
        L.lsm_refined_nodes.argtypes = [I32, I64, P, P, P, ctypes.POINTER(I64)]
        L.lsm_solve_charts_nodes.argtypes = [P, I64, P, P, D, I32, I32, P, P, P, ctypes.POINTER(_Stats), P]
        L.lsm_chart_frames_nodes.argtypes = [P, I64, P, P, P, P, P, P, P, P]
        L.lsm_gauss_flux_nodes.argtypes = [P, I64, P, P, P, P, P, P, P, P]
        L.lsm_gauss_flux.argtypes = [P, I32, P, P, P, P, P, P]
        L.lsm_flux_per_triangle.argtypes = [P, I64, P, P, P, P, P, P, P, P]
        L.lsm_refine_adaptive.argtypes = [P, I32, D, D, I32, P, P, ctypes.POINTER(ctypes.c_int), P]
        L.lsm_check_error.argtypes = [P, P]
        L.lsm_test_inject_wait_timeout.argtypes = [P, I32]
        L.lsm_measure_peaks.argtypes = [P, ctypes.POINTER(_Peaks), P]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
        _lib = L
        return L


def lib():
    return load()


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _as(a, dtype):
    """Contiguous array of the requested dtype on the same side as `a`."""
    if _is_torch(a):
        import torch
        td = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        return a.to(td).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def refined_nodes(order: int, levels):
    """Chart nodes of triangles refined 1 -> 4 levels[j] times (lsm_refined_nodes,
    host only): (tri [N], uvw [N, 3]) in the parents' coordinates."""
    L = load()
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    n = ctypes.c_int64()
    rc = L.lsm_refined_nodes(int(order), int(lv.shape[0]), _ptr(lv), None, None, ctypes.byref(n))
    if rc != 0:
        raise LsmError(rc, "lsm_refined_nodes: bad order or levels (0..4)")
    tri, uvw = np.empty(n.value, dtype=np.int32), np.empty((n.value, 3))
    rc = L.lsm_refined_nodes(int(order), int(lv.shape[0]), _ptr(lv), _ptr(tri), _ptr(uvw), ctypes.byref(n))
    if rc != 0:
        raise LsmError(rc, "lsm_refined_nodes failed")
    return tri, uvw


class Context:
    """A library context on one CUDA device (lsm_create)."""

    def __init__(self, device: int = 0, cutoff_fp64: float = 0.0, cutoff_mixed: float = 0.0,
                 mixed_switch: float = 0.0, mixed_accept: float = 0.0, tree_degree: int = 0,
                 tree_theta: float = 0.0, tree_min_sources: int = 0, tree_ff_degree: int = 0,
                 tree_ff_theta: float = 0.0, tree_ff_min_sources: int = 0, tree_grid: int = 0,
                 tree_ff_cluster: int = 0, tree_cluster: int = 0, ff_block: int = 0, mixed_block: int = 0,
                 newton_tree_degree: int = 0, newton_tree_theta: float = 0.0, newton_cutoff: float = 0.0):
        """Zero selects a default.  tree_*: the treecode far field of the mixed
        path (Chebyshev degree, opening parameter, and the source count from
        which a mesh uses it; tree_min_sources=-1 turns it off); tree_ff_*: the
        same for the float-float path.  tree_grid: 1 oriented per-axis proxy
        grids with a degree ladder (the default), 2 full (degree + 1)^3
        axis-aligned grids of one degree.  tree_ff_cluster: targets per target
        cluster of the float-float treecode (0: 4096, -1: off); tree_cluster:
        the same for the mixed treecode (0: 4096, -1: off).  ff_block:
        targets per CTA of the float-float kernel (64, the default, or 128).
        mixed_block: targets per CTA of the mixed kernel (64, 128 or 256; 0:
        the autotuner's choice, else 64).  newton_tree_degree/theta: the
        coarser mixed treecode of a chart solve's mixed Newton sweeps (0: 5
        and 0.5; degree -1: the mesh's mixed treecode); newton_cutoff: their
        near-field radius in sigma (0: 5.0)."""
        self._L = load()
        opt = _Options(cutoff_fp64, cutoff_mixed, mixed_switch, mixed_accept, int(tree_degree),
                       float(tree_theta), int(tree_min_sources), int(tree_ff_degree), float(tree_ff_theta),
                       int(tree_ff_min_sources), int(tree_grid), int(tree_ff_cluster), int(tree_cluster), int(ff_block),
                       int(mixed_block), int(newton_tree_degree), float(newton_tree_theta), float(newton_cutoff))
        h = ctypes.c_void_p()
        rc = self._L.lsm_create(ctypes.byref(h), int(device), ctypes.byref(opt))
        if rc != 0:
            raise LsmError(rc, "lsm_create failed (no CUDA device?)")
        self._h = h
        self.device = device

    def _check(self, rc):
        if rc != 0:
            raise LsmError(rc, self._L.lsm_last_error(self._h).decode(errors="replace"))

    @property
    def launch_count(self) -> int:
        return int(self._L.lsm_launch_count(self._h))

    def set_profiling(self, enable: bool = True):
        """Time every pair-kernel launch with CUDA events on its stream."""
        self._check(self._L.lsm_set_profiling(self._h, 1 if enable else 0))

    def read_stats(self, reset: bool = False) -> dict:
        """Launch count, pairs evaluated (near / far tiles) and pair-kernel time."""
        st = _CtxStats()
        self._check(self._L.lsm_read_stats(self._h, ctypes.byref(st), 1 if reset else 0))
        out = {}
        for k, _ in _CtxStats._fields_:
            v = getattr(st, k)
            out[k] = list(v) if k.startswith("kind_") else v
        return out

    def check_error(self, stream=None):
        """Raise LsmError (TIMEOUT) if a pair kernel this thread launched gave
        up on a bounded wait since the last check (lsm_check_error)."""
        self._check(self._L.lsm_check_error(self._h, _stream_handle(stream)))

    def inject_wait_timeout(self, enable: bool = True):
        """Test hook (lsm_test_inject_wait_timeout): pair kernels arm their
        first stage without a copy, so that their bounded wait runs out."""
        self._check(self._L.lsm_test_inject_wait_timeout(self._h, 1 if enable else 0))

    def measure_peaks(self, stream=None) -> dict:
        """Measured FP32 (scalar and packed), FP64 FMA and special-function
        throughput of this GPU (lsm_measure_peaks)."""
        p = _Peaks()
        self._check(self._L.lsm_measure_peaks(self._h, ctypes.byref(p), _stream_handle(stream)))
        out = {k: getattr(p, k) for k, _ in _Peaks._fields_ if k != "ms"}
        out["ms"] = list(p.ms)
        return out

    def upload(self, verts, tris, sigma=None, n_gl: int = 4, subdiv: int = 0, stream=None) -> "Mesh":
        return Mesh(self, verts, tris, sigma, n_gl, subdiv, stream)

    def upload_quadratic(self, verts, tris6, sigma=None, n_gl: int = 4, subdiv: int = 0, stream=None) -> "Mesh":
        """A skeleton of 6-node quadratic patches (lsm_mesh_upload_quadratic)."""
        t = _as(tris6, np.int32)
        if t.ndim != 2 or t.shape[1] != 6:
            raise ValueError("tris6 must be [m, 6]")
        return Mesh(self, verts, t, sigma, n_gl, subdiv, stream)

    def upload_sigma_x(self, verts, tris, lam: float = 0.0, sigma0: float = 0.0, n_gl: int = 4, subdiv: int = 0,
                       stream=None) -> "Mesh":
        """A mesh with the target-dependent sigma(x) of eq. sigma2."""
        return Mesh(self, verts, tris, None, n_gl, subdiv, stream, sigma_x=True, lam=lam, sigma0=sigma0)

    def close(self):
        if getattr(self, "_h", None):
            self._L.lsm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Resident device state of one skeleton triangulation (lsm_mesh_upload)."""

    def __init__(self, ctx: Context, verts, tris, sigma=None, n_gl: int = 4, subdiv: int = 0,
                 stream=None, sigma_x: bool = False, lam: float = 0.0, sigma0: float = 0.0):
        """sigma_x=True: target-dependent sigma(x) (lsm_mesh_upload_sigmax, with
        lambda and sigma0, 0 for the defaults); else per-triangle sigma.
        tris [m, 6]: quadratic patches (lsm_mesh_upload_quadratic)."""
        self.ctx = ctx
        v = _as(verts, np.float64)
        t = _as(tris, np.int32)
        q = _Quad(int(n_gl), int(subdiv))
        h = ctypes.c_void_p()
        if sigma_x:
            rc = ctx._L.lsm_mesh_upload_sigmax(ctx._h, _ptr(v), int(v.shape[0]), _ptr(t), int(t.shape[0]),
                                               float(lam), float(sigma0), ctypes.byref(q),
                                               _stream_handle(stream), ctypes.byref(h))
        elif t.shape[1] == 6:
            s = _as(sigma, np.float64) if sigma is not None else None
            rc = ctx._L.lsm_mesh_upload_quadratic(ctx._h, _ptr(v), int(v.shape[0]), _ptr(t), int(t.shape[0]),
                                                  _ptr(s), ctypes.byref(q), _stream_handle(stream), ctypes.byref(h))
        else:
            s = _as(sigma, np.float64) if sigma is not None else None
            rc = ctx._L.lsm_mesh_upload(ctx._h, _ptr(v), int(v.shape[0]), _ptr(t), int(t.shape[0]),
                                        _ptr(s), ctypes.byref(q), _stream_handle(stream), ctypes.byref(h))
        ctx._check(rc)
        self._h = h
        self.n_triangles = int(t.shape[0])

    def eval_sigma(self, x, stream=None):
        """sigma(x) [n] and grad sigma [n, 3] of a sigma(x) mesh (lsm_eval_sigma)."""
        xs = _as(x, np.float64)
        n = int(xs.shape[0])
        if _is_torch(xs):
            import torch
            sg = torch.empty(n, dtype=torch.float64, device=xs.device)
            gs = torch.empty((n, 3), dtype=torch.float64, device=xs.device)
        else:
            sg, gs = np.empty(n), np.empty((n, 3))
        rc = self.ctx._L.lsm_eval_sigma(self._h, _ptr(xs), n, _ptr(sg), _ptr(gs), _stream_handle(stream))
        self.ctx._check(rc)
        return sg, gs

    @property
    def sigma0(self) -> float:
        """sigma0 of a sigma(x) mesh (0 otherwise)."""
        out = ctypes.c_double()
        self.ctx._check(self.ctx._L.lsm_mesh_get_sigma0(self._h, ctypes.byref(out)))
        return out.value

    def info(self) -> dict:
        inf = _Info()
        self.ctx._check(self.ctx._L.lsm_mesh_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _Info._fields_}

    def eval_phi_grad(self, x, precision: int = FP64, phi=None, grad=None, with_grad: bool = True,
                      stream=None):
        """Phi and grad Phi at targets x [n, 3] (lsm_eval_phi_grad)."""
        xs = _as(x, np.float64)
        n = int(xs.shape[0])
        if phi is None:
            if _is_torch(xs):
                import torch
                phi = torch.empty(n, dtype=torch.float64, device=xs.device)
                if with_grad and grad is None:
                    grad = torch.empty((n, 3), dtype=torch.float64, device=xs.device)
            else:
                phi = np.empty(n)
                if with_grad and grad is None:
                    grad = np.empty((n, 3))
        rc = self.ctx._L.lsm_eval_phi_grad(self._h, _ptr(xs), n, _ptr(phi), _ptr(grad), int(precision),
                                           _stream_handle(stream))
        self.ctx._check(rc)
        return phi, grad

    def autotune(self, x, err_budget: float = 5e-8, stream=None) -> dict:
        """Choose this mesh's mixed-path far field (direct, or the treecode's
        degree and opening parameter), then its near-field radius and target
        tile, on a sample of the targets x [n, 3] (lsm_autotune).  Returns the
        choice and the measured time and error."""
        xs = _as(x, np.float64)
        r = _TuneResult()
        rc = self.ctx._L.lsm_autotune(self._h, _ptr(xs), int(xs.shape[0]), float(err_budget), ctypes.byref(r),
                                      _stream_handle(stream))
        self.ctx._check(rc)
        return {k: getattr(r, k) for k, _ in _TuneResult._fields_ if k != "reserved"}

    def chart_frames(self, order: int, h, grad, stream=None):
        """Local coordinates x_u, x_v [N, 3] and |x_u x x_v| [N] of the solved
        charts from their h [N] and grad Phi [N, 3] (lsm_chart_frames); torch
        inputs give device-resident torch outputs."""
        hs, gs = _as(h, np.float64), _as(grad, np.float64)
        n = int(hs.shape[0])
        if _is_torch(hs):
            import torch
            xu = torch.empty((n, 3), dtype=torch.float64, device=hs.device)
            xv = torch.empty((n, 3), dtype=torch.float64, device=hs.device)
            jac = torch.empty(n, dtype=torch.float64, device=hs.device)
        else:
            xu, xv, jac = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        rc = self.ctx._L.lsm_chart_frames(self._h, int(order), _ptr(hs), _ptr(gs), _ptr(xu), _ptr(xv), _ptr(jac),
                                          _stream_handle(stream))
        self.ctx._check(rc)
        return xu, xv, jac

    def solve_charts_nodes(self, tri, uvw, tol: float = 1e-12, max_iter: int = 20, precision: int = FP64,
                           device_out: bool = False, stream=None):
        """Charts at explicit nodes (lsm_solve_charts_nodes): (x, h, status, SolveStats);
        with device_out the outputs are CUDA tensors on the mesh's device."""
        t, u = _as(tri, np.int32), _as(uvw, np.float64)
        n = int(t.shape[0])
        if device_out:
            import torch
            dev = torch.device("cuda", self.ctx.device)
            x = torch.empty((n, 3), dtype=torch.float64, device=dev)
            h = torch.empty(n, dtype=torch.float64, device=dev)
            st = torch.empty(n, dtype=torch.int32, device=dev)
        else:
            x, h, st = np.empty((n, 3)), np.empty(n), np.empty(n, dtype=np.int32)
        stats = _Stats()
        rc = self.ctx._L.lsm_solve_charts_nodes(self._h, n, _ptr(t), _ptr(u), float(tol), int(max_iter),
                                                int(precision), _ptr(x), _ptr(h), _ptr(st), ctypes.byref(stats),
                                                _stream_handle(stream))
        self.ctx._check(rc)
        return x, h, st, _stats(stats)

    def chart_frames_nodes(self, tri, uvw, h, grad, stream=None):
        t, u = _as(tri, np.int32), _as(uvw, np.float64)
        hs, gs = _as(h, np.float64), _as(grad, np.float64)
        n = int(t.shape[0])
        xu, xv, jac = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
        rc = self.ctx._L.lsm_chart_frames_nodes(self._h, n, _ptr(t), _ptr(u), _ptr(hs), _ptr(gs), _ptr(xu), _ptr(xv),
                                                _ptr(jac), _stream_handle(stream))
        self.ctx._check(rc)
        return xu, xv, jac

    def gauss_flux_nodes(self, tri, uvw, x, grad, jac, x0, stream=None) -> float:
        t, u = _as(tri, np.int32), _as(uvw, np.float64)
        xs, gs, js = _as(x, np.float64), _as(grad, np.float64), _as(jac, np.float64)
        p0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(3))
        out = ctypes.c_double()
        rc = self.ctx._L.lsm_gauss_flux_nodes(self._h, int(t.shape[0]), _ptr(t), _ptr(u), _ptr(xs), _ptr(gs), _ptr(js),
                                              _ptr(p0), ctypes.byref(out), _stream_handle(stream))
        self.ctx._check(rc)
        return out.value

    def flux_per_triangle(self, tri, uvw, x, grad, jac, x0, stream=None):
        """Gauss flux split by skeleton triangle (lsm_flux_per_triangle), host [m]."""
        t, u = _as(tri, np.int32), _as(uvw, np.float64)
        xs, gs, js = _as(x, np.float64), _as(grad, np.float64), _as(jac, np.float64)
        p0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(3)
        out = np.empty(self.n_triangles)
        rc = self.ctx._L.lsm_flux_per_triangle(self._h, int(t.shape[0]), _ptr(t), _ptr(u), _ptr(xs), _ptr(gs),
                                               _ptr(js), _ptr(p0), _ptr(out), _stream_handle(stream))
        self.ctx._check(rc)
        return out

    def refine_adaptive(self, order: int, flux_tol: float, max_level: int, x0, newton_tol: float = 1e-12,
                        stream=None):
        """Per-triangle refinement levels from the a posteriori flux estimate
        (lsm_refine_adaptive): (levels [m], rounds)."""
        p0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(3)
        lv = np.zeros(self.n_triangles, dtype=np.int32)
        rounds = ctypes.c_int()
        rc = self.ctx._L.lsm_refine_adaptive(self._h, int(order), float(newton_tol), float(flux_tol), int(max_level),
                                             _ptr(p0), _ptr(lv), ctypes.byref(rounds), _stream_handle(stream))
        self.ctx._check(rc)
        return lv, int(rounds.value)

    def eval_hessian(self, x, stream=None):
        """Hessian of Phi [n, 6] = (xx, xy, xz, yy, yz, zz) at targets x [n, 3]
        (lsm_eval_hessian)."""
        xs = _as(x, np.float64)
        n = int(xs.shape[0])
        if _is_torch(xs):
            import torch
            hs = torch.empty((n, 6), dtype=torch.float64, device=xs.device)
        else:
            hs = np.empty((n, 6))
        rc = self.ctx._L.lsm_eval_hessian(self._h, _ptr(xs), n, _ptr(hs), _stream_handle(stream))
        self.ctx._check(rc)
        return hs

    def chart_curvature(self, order: int, h, grad, hess, stream=None):
        """Second derivatives x_uu, x_uv, x_vv [N, 3] of the solved charts and the
        mean (sum of principal curvatures) and Gaussian curvatures [N] at their
        nodes (lsm_chart_curvature)."""
        hs, gs, ss = _as(h, np.float64), _as(grad, np.float64), _as(hess, np.float64)
        n = int(hs.shape[0])
        if _is_torch(hs):
            import torch
            mk = lambda *sh: torch.empty(sh, dtype=torch.float64, device=hs.device)
        else:
            mk = lambda *sh: np.empty(sh)
        uu, uv, vv, km, kg = mk(n, 3), mk(n, 3), mk(n, 3), mk(n), mk(n)
        rc = self.ctx._L.lsm_chart_curvature(self._h, int(order), _ptr(hs), _ptr(gs), _ptr(ss), _ptr(uu), _ptr(uv),
                                             _ptr(vv), _ptr(km), _ptr(kg), _stream_handle(stream))
        self.ctx._check(rc)
        return uu, uv, vv, km, kg

    def gauss_flux(self, order: int, x, grad, jac, x0, stream=None) -> float:
        """Gauss flux error eps0 of the charts about x0 (lsm_gauss_flux)."""
        xs, gs, js = _as(x, np.float64), _as(grad, np.float64), _as(jac, np.float64)
        p0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).reshape(3))
        out = ctypes.c_double()
        rc = self.ctx._L.lsm_gauss_flux(self._h, int(order), _ptr(xs), _ptr(gs), _ptr(js), _ptr(p0),
                                        ctypes.byref(out), _stream_handle(stream))
        self.ctx._check(rc)
        return out.value

    def solve_charts(self, order: int = 8, tol: float = 1e-12, max_iter: int = 20,
                     precision: int = FP64, device_out: bool = False, stream=None):
        """Chart nodes on Phi = 1/2 by Newton's method (lsm_solve_charts).
        Returns (x [N,3], h [N], status [N], SolveStats)."""
        n_gl = order // 2 + 2
        N = self.n_triangles * n_gl * n_gl
        if device_out:
            import torch
            dev = torch.device("cuda", self.ctx.device)
            x = torch.empty((N, 3), dtype=torch.float64, device=dev)
            h = torch.empty(N, dtype=torch.float64, device=dev)
            st = torch.empty(N, dtype=torch.int32, device=dev)
        else:
            x, h, st = np.empty((N, 3)), np.empty(N), np.empty(N, dtype=np.int32)
        stats = _Stats()
        rc = self.ctx._L.lsm_solve_charts(self._h, int(order), float(tol), int(max_iter), int(precision),
                                          _ptr(x), _ptr(h), _ptr(st), ctypes.byref(stats),
                                          _stream_handle(stream))
        self.ctx._check(rc)
        return x, h, st, _stats(stats)

    def free(self):
        if getattr(self, "_h", None):
            # a closed context has freed its meshes already (lsm_destroy)
            if getattr(self.ctx, "_h", None):
                self.ctx._L.lsm_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _stats(st: "_Stats") -> SolveStats:
    return SolveStats(st.iterations, st.n_nodes, st.n_converged, st.n_failed, st.eps_newton, st.max_residual,
                      st.evals_fp32, st.evals_fp64, list(st.active_per_iter)[:max(min(st.iterations, 32), 0)],
                      st.evals_near_only)


class Batch:
    """Many uploaded meshes solved together (lsm_batch_create)."""

    def __init__(self, ctx: Context, meshes, stream=None):
        self.ctx = ctx
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = ctypes.c_void_p()
        ctx._check(ctx._L.lsm_batch_create(ctx._h, arr, len(self.meshes), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n_triangles = sum(m.n_triangles for m in self.meshes)

    def solve_charts(self, order: int = 6, tol: float = 1e-10, max_iter: int = 20, precision: int = MIXED,
                     use_graph: bool = True, device_out: bool = False, stream=None):
        """Chart nodes of every mesh (lsm_batch_solve_charts), concatenated in mesh order."""
        n_gl = order // 2 + 2
        N = self.n_triangles * n_gl * n_gl
        if device_out:
            import torch
            dev = torch.device("cuda", self.ctx.device)
            x = torch.empty((N, 3), dtype=torch.float64, device=dev)
            h = torch.empty(N, dtype=torch.float64, device=dev)
            st = torch.empty(N, dtype=torch.int32, device=dev)
        else:
            x, h, st = np.empty((N, 3)), np.empty(N), np.empty(N, dtype=np.int32)
        stats = _Stats()
        rc = self.ctx._L.lsm_batch_solve_charts(self._h, int(order), float(tol), int(max_iter), int(precision),
                                                1 if use_graph else 0, _ptr(x), _ptr(h), _ptr(st),
                                                ctypes.byref(stats), _stream_handle(stream))
        self.ctx._check(rc)
        return x, h, st, _stats(stats)

    def autotune(self, order: int = 6, err_budget: float = 5e-8, stream=None) -> dict:
        """Mixed-kernel near-field radius and target tile for this batch
        (lsm_batch_autotune), measured on a sample of its meshes' nodes."""
        r = _TuneResult()
        self.ctx._check(self.ctx._L.lsm_batch_autotune(self._h, int(order), float(err_budget), ctypes.byref(r),
                                                        _stream_handle(stream)))
        return {k: getattr(r, k) for k, _ in _TuneResult._fields_ if k != "reserved"}

    def free(self):
        if getattr(self, "_h", None):
            if getattr(self.ctx, "_h", None):
                self.ctx._L.lsm_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (lsm_server_*): requests are admitted
    in arrival order as worker slots and HBM budget free up, and run
    concurrently on their slots' streams."""

    def __init__(self, ctx: Context, slots: int = 4, hbm_budget_bytes: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(ctx._L.lsm_server_create(ctx._h, int(slots), int(hbm_budget_bytes), ctypes.byref(h)))
        self._h = h

    def submit(self, verts, tris, sigma=None, n_gl: int = 4, subdiv: int = 0, order: int = 8,
               tol: float = 1e-10, max_iter: int = 20, precision: int = MIXED) -> int:
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        s = np.ascontiguousarray(sigma, dtype=np.float64) if sigma is not None else None
        rq = _Request(v.ctypes.data, len(v), t.ctypes.data, len(t), s.ctypes.data if s is not None else None,
                      _Quad(int(n_gl), int(subdiv)), int(order), float(tol), int(max_iter), int(precision))
        tk = ctypes.c_int64()
        self.ctx._check(self.ctx._L.lsm_server_submit(self._h, ctypes.byref(rq), ctypes.byref(tk)))
        return int(tk.value)

    def result(self, ticket: int, wait: bool = True, release: bool = True):
        """The finished request as a dict (arrays copied), or None while pending."""
        r = _Result()
        rc = self.ctx._L.lsm_server_poll(self._h, int(ticket), 1 if wait else 0, ctypes.byref(r))
        if rc == 1:
            return None
        self.ctx._check(rc)
        n = int(r.n_nodes)
        out = {"status": int(r.status), "n_nodes": n, "t_submit_ms": r.t_submit_ms, "t_start_ms": r.t_start_ms,
               "t_done_ms": r.t_done_ms, "device_bytes": int(r.device_bytes), "stats": _stats(r.stats),
               "error": (r.error or b"").decode(errors="replace")}
        if r.status == 0 and n > 0:
            out["x"] = np.ctypeslib.as_array(r.x, shape=(n, 3)).copy()
            out["h"] = np.ctypeslib.as_array(r.h, shape=(n,)).copy()
            out["node_status"] = np.ctypeslib.as_array(r.node_status, shape=(n,)).copy()
        if release:
            self.ctx._L.lsm_server_release(self._h, int(ticket))
        return out

    def cancel(self, ticket: int) -> bool:
        """Take a still-queued request off the queue (lsm_server_cancel);
        False when it has already started or finished."""
        return self.ctx._L.lsm_server_cancel(self._h, int(ticket)) == 0

    def info(self) -> dict:
        inf = _ServerInfo()
        self.ctx._check(self.ctx._L.lsm_server_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _ServerInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self.ctx, "_h", None):
                self.ctx._L.lsm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
