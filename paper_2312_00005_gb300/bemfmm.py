"""Thin ctypes binding of the C ABI in ``include/bemfmm.h``.

Argument marshalling only: every step of the BEM + FMM path runs in the CUDA
library ``_bemfmm.so`` built from ``csrc/``.  PyTorch supplies device memory
(complex64 CUDA tensors) and streams.  Importing this module loads the
library and raises if it is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "VELO", "PRES", "ADMI", "MODE_FMM", "MODE_DIRECT", "BemError", "Params", "Medium", "Source",
    "SolveInfo", "PlanStats", "Mesh", "lib", "launch_count", "plane_wave", "point_source", "timing_enable",
    "timing_get", "plan_stats_host", "mesh_check_host", "default_params", "admittance_loss",
]

VELO, PRES, ADMI = 0, 1, 2
MODE_FMM, MODE_DIRECT = 0, 1
SRC_PLANE, SRC_POINT = 0, 1
OK, W_NOT_CONVERGED, W_UNDERRESOLVED = 0, 1, 2
E_SUBDIV_LIMIT = -2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_bemfmm.so")


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bemfmm error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("quad_tol", ctypes.c_double), ("m_max", ctypes.c_int32),
        ("rt_subdiv", ctypes.c_double), ("max_depth", ctypes.c_int32), ("trunc_factor", ctypes.c_double),
        ("L_min", ctypes.c_int32), ("admissibility", ctypes.c_double), ("leaf_edge", ctypes.c_double),
        ("stability_max", ctypes.c_double), ("near_store", ctypes.c_int32), ("restart", ctypes.c_int32),
        ("autotune", ctypes.c_int32), ("tau", ctypes.c_double), ("row_scaling", ctypes.c_int32),
        ("check_orientation", ctypes.c_int32), ("symmetric_far", ctypes.c_int32),
        ("block_jacobi", ctypes.c_int32), ("far_precision", ctypes.c_int32), ("near_chunk", ctypes.c_int32),
        ("gs_rows", ctypes.c_int32), ("field_mode", ctypes.c_int32), ("far_table", ctypes.c_int32),
        ("graphs", ctypes.c_int32), ("near_transpose", ctypes.c_int32),
    ]


class Medium(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("rho", ctypes.c_double)]


class Source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("vec", ctypes.c_double * 3), ("amp", ctypes.c_double * 2)]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("relres", ctypes.c_double),
        ("seconds", ctypes.c_double), ("levels", ctypes.c_int32), ("L", ctypes.c_int32 * 16),
        ("near_nnz", ctypes.c_int64), ("status", ctypes.c_int32), ("setup_seconds", ctypes.c_double),
        ("rhs_seconds", ctypes.c_double), ("gmres_seconds", ctypes.c_double),
    ]


class PlanStats(ctypes.Structure):
    _fields_ = [
        ("n_elements", ctypes.c_int64), ("leaf_level", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("level_depth", ctypes.c_int32 * 16), ("L", ctypes.c_int32 * 16), ("n_clusters", ctypes.c_int32 * 16),
        ("n_interactions", ctypes.c_int64 * 16), ("n_offsets", ctypes.c_int32 * 16), ("n_leaves", ctypes.c_int32),
        ("near_nnz", ctypes.c_int64), ("near_quad_points", ctypes.c_int64), ("leaf_edge", ctypes.c_double),
        ("mean_edge", ctypes.c_double), ("device_bytes", ctypes.c_int64), ("far_pairs", ctypes.c_int64),
        ("n_tuned", ctypes.c_int32), ("tuned_depth", ctypes.c_int32 * 4), ("tuned_seconds", ctypes.c_double * 4),
        ("asymmetric_pairs", ctypes.c_int64), ("order_R", ctypes.c_double * 8),
        ("near_light_entries", ctypes.c_int64), ("near_light_points", ctypes.c_int64),
        ("near_heavy_entries", ctypes.c_int64), ("near_heavy_points", ctypes.c_int64),
        ("n_src_elements", ctypes.c_int64 * 16), ("n_tgt_elements", ctypes.c_int64 * 16),
        ("asymmetric_near_pairs", ctypes.c_int64),
    ]

    def as_dict(self):
        n = self.levels
        return {
            "n_elements": self.n_elements, "leaf_level": self.leaf_level, "levels": n,
            "level_depth": list(self.level_depth[:n]), "L": list(self.L[:n]),
            "n_clusters": list(self.n_clusters[:n]), "n_interactions": list(self.n_interactions[:n]),
            "n_offsets": list(self.n_offsets[:n]), "n_leaves": self.n_leaves, "near_nnz": self.near_nnz,
            "near_quad_points": self.near_quad_points, "leaf_edge": self.leaf_edge,
            "mean_edge": self.mean_edge, "device_bytes": self.device_bytes, "far_pairs": self.far_pairs,
            "asymmetric_pairs": self.asymmetric_pairs, "order_R": list(self.order_R),
            "near_light_entries": self.near_light_entries, "near_light_points": self.near_light_points,
            "near_heavy_entries": self.near_heavy_entries, "near_heavy_points": self.near_heavy_points,
            "n_src_elements": list(self.n_src_elements[:n]), "n_tgt_elements": list(self.n_tgt_elements[:n]),
            "asymmetric_near_pairs": self.asymmetric_near_pairs,
            "autotune": [(self.tuned_depth[q], self.tuned_seconds[q]) for q in range(self.n_tuned)],
        }


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError("bemfmm CUDA library not built (%s missing): run "
                              "`python -m paper_2312_00005_gb300.build`" % _SO)
        L = ctypes.CDLL(_SO)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "bem_params_default": (None, [ctypes.POINTER(Params)]),
            "bem_mesh_create": (ctypes.c_int, [P, i64, P, i64, P, P, P, ctypes.POINTER(Params), ctypes.POINTER(P)]),
            "bem_mesh_destroy": (ctypes.c_int, [P]),
            "bem_matvec": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, P, P, i32, P]),
            "bem_matvec_host": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, P, P, i32, P]),
            "bem_matvec_transpose": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, P, P, P]),
            "bem_solve": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, ctypes.POINTER(Source), i32, d, i32,
                                         P, P, ctypes.POINTER(SolveInfo), P]),
            "bem_evaluate": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), ctypes.POINTER(Source), i32, P, P, P,
                                            i64, P, P]),
            "bem_solve_multi": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, ctypes.POINTER(Source), i32, d,
                                               i32, P, P, ctypes.POINTER(SolveInfo), P]),
            "bem_solve_sweep": (ctypes.c_int, [P, P, i32, ctypes.POINTER(Medium), P, i32, ctypes.POINTER(Source), i32,
                                               d, i32, P, P, P, i64, P, ctypes.POINTER(SolveInfo), P]),
            "bem_evaluate_velocity": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), ctypes.POINTER(Source), i32, P,
                                                     P, P, i64, P, P]),
            "bem_admittance_gradient": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P, i32, ctypes.POINTER(Source),
                                                       i32, P, i64, d, i32, P, P, ctypes.POINTER(d), P,
                                                       ctypes.POINTER(SolveInfo), P]),
            "bem_mesh_stats": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), ctypes.POINTER(PlanStats)]),
            "bem_mesh_check_host": (ctypes.c_int, [P, i64, P, i64, ctypes.POINTER(d), ctypes.POINTER(i64),
                                                   ctypes.POINTER(i64)]),
            "bem_field_plan_stats_host": (ctypes.c_int, [P, i64, P, i64, P, i64, ctypes.POINTER(Params), d, d,
                                                         ctypes.POINTER(FieldStats)]),
            "bem_plan_stats_host": (ctypes.c_int, [P, i64, P, i64, ctypes.POINTER(Params), d, d,
                                                   ctypes.POINTER(PlanStats)]),
            "bem_mesh_release_plan": (ctypes.c_int, [P]),
            "bem_mesh_blocks": (ctypes.c_int, [P, d, ctypes.POINTER(Medium), P]),
            "bem_timing_enable": (ctypes.c_int, [ctypes.c_int]),
            "bem_timing_get": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64)]),
            "bem_selftest_sincos": (ctypes.c_int, [P, i64, P, P]),
            "bem_matvec_direct_noalloc": (ctypes.c_int, [P, i64, P, i64, d, ctypes.POINTER(Medium), P, P, P]),
            "bem_test_hooks": (ctypes.c_int, [i64, ctypes.POINTER(i64)]),
            "bem_krylov_basis": (ctypes.c_int, [P, i32, P, i32, ctypes.POINTER(i32)]),
            "bem_launch_count": (ctypes.c_uint64, []),
            "bem_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def test_hooks(alloc_fail_after=-1) -> int:
    """Set the allocation-failure test hook (see bem_test_hooks in the
    header); returns the bytes the library holds in device allocations."""
    live = ctypes.c_int64(0)
    _check(lib().bem_test_hooks(int(alloc_fail_after), ctypes.byref(live)))
    return live.value


def launch_count() -> int:
    return int(lib().bem_launch_count())


def timing_enable(flag: bool) -> None:
    """Per-kernel CUDA-event timing on the library's stream (see the header)."""
    lib().bem_timing_enable(1 if flag else 0)


def timing_get(name: str):
    """(total milliseconds, launches) recorded for kernel `name`."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    code = lib().bem_timing_get(name.encode(), ctypes.byref(ms), ctypes.byref(n))
    if code != 0:
        return 0.0, 0
    return ms.value, n.value


def selftest_sincos(x):
    """(fast sin, fast cos, sincospif sin, sincospif cos) of 2 pi x for a float32
    CUDA tensor x of phases in turns."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    out = torch.empty((x.numel(), 4), dtype=torch.float32, device=x.device)
    _check(lib().bem_selftest_sincos(ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(out.data_ptr()),
                                     _stream_ptr(None)))
    return out


def matvec_direct_noalloc(nodes_dev, tris_dev, freq, x, y, c=343.0, rho=1.21, stream=None):
    """Direct sound-hard product that allocates no device memory (see the
    header): nodes_dev float64 [n_nodes, 3], tris_dev int32 [n, 3], x and y
    complex64 [n], all contiguous CUDA tensors on the current device, owned
    by the caller.  The C entry point cannot see the tensors' shapes, so they
    are checked here: a wrong shape would make its kernels read past the
    caller's buffers."""
    import torch
    for name, t, dt in (("nodes_dev", nodes_dev, torch.float64), ("tris_dev", tris_dev, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("%s must be a contiguous %s CUDA tensor" % (name, dt))
        if t.dim() != 2 or t.shape[1] != 3:
            raise ValueError("%s must have shape [*, 3], got %s" % (name, tuple(t.shape)))
    n = tris_dev.shape[0]
    for name, t in (("x", x), ("y", y)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
            raise TypeError("%s must be a contiguous complex64 CUDA tensor" % name)
        if t.numel() != n:
            raise ValueError("%s has %d elements, the mesh %d triangles" % (name, t.numel(), n))
    dev = torch.cuda.current_device()
    for name, t in (("nodes_dev", nodes_dev), ("tris_dev", tris_dev), ("x", x), ("y", y)):
        if t.device.index != dev:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, t.device.index, dev))
    med = Medium(float(c), float(rho))
    return _check(lib().bem_matvec_direct_noalloc(ctypes.c_void_p(nodes_dev.data_ptr()), nodes_dev.shape[0],
                                                  ctypes.c_void_p(tris_dev.data_ptr()), n, float(freq),
                                                  ctypes.byref(med), _dptr(x, n), _dptr(y, n), _stream_ptr(stream)))


def _check(code, allow_warn=True):
    if code < 0 or (code > 0 and not allow_warn):
        raise BemError(code, lib().bem_last_error().decode(errors="replace"))
    return code


def default_params(**kw) -> Params:
    p = Params()
    lib().bem_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def plane_wave(direction=(0.0, 0.0, 1.0), amp=1.0 + 0.0j) -> Source:
    s = Source()
    s.kind = SRC_PLANE
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    s.vec[:] = list(d)
    s.amp[:] = [complex(amp).real, complex(amp).imag]
    return s


def point_source(position, amp=1.0 + 0.0j) -> Source:
    s = Source()
    s.kind = SRC_POINT
    s.vec[:] = [float(v) for v in position]
    s.amp[:] = [complex(amp).real, complex(amp).imag]
    return s


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
        raise TypeError("expected a contiguous complex64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError("tensor too small: %d < %d" % (t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def _admittance(adm):
    if adm is None:
        return None, 0
    a = np.asarray(adm, dtype=np.complex128).reshape(-1)
    buf = np.ascontiguousarray(np.stack([a.real, a.imag], axis=1))
    return buf, a.shape[0]


def mesh_check_host(nodes, tris) -> dict:
    """Orientation diagnostics of a closed surface (host only): signed
    enclosed volume (positive for normals out of the volume), open edges,
    inconsistently wound edges."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    vol, op, mis = ctypes.c_double(0.0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().bem_mesh_check_host(nodes.ctypes.data_as(ctypes.c_void_p), nodes.shape[0],
                                     tris.ctypes.data_as(ctypes.c_void_p), tris.shape[0], ctypes.byref(vol),
                                     ctypes.byref(op), ctypes.byref(mis)))
    return {"volume": vol.value, "open_edges": op.value, "misoriented_edges": mis.value}


def plan_stats_host(nodes, tris, freq, c=343.0, params=None) -> dict:
    """Clustering and near / interaction lists for a frequency, built on the
    host only (no GPU needed)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    p = params if params is not None else default_params()
    st = PlanStats()
    _check(lib().bem_plan_stats_host(nodes.ctypes.data_as(ctypes.c_void_p), nodes.shape[0],
                                     tris.ctypes.data_as(ctypes.c_void_p), tris.shape[0], ctypes.byref(p),
                                     float(freq), float(c), ctypes.byref(st)))
    return st.as_dict()


class FieldStats(ctypes.Structure):
    _fields_ = [
        ("leaf_level", ctypes.c_int32), ("levels", ctypes.c_int32), ("level_depth", ctypes.c_int32 * 16),
        ("L", ctypes.c_int32 * 16), ("n_point_clusters", ctypes.c_int32 * 16),
        ("n_interactions", ctypes.c_int64 * 16), ("n_offsets", ctypes.c_int32 * 16),
        ("near_pairs", ctypes.c_int64), ("far_pairs", ctypes.c_int64), ("n_point_leaves", ctypes.c_int64),
    ]

    def as_dict(self):
        n = self.levels
        return {"leaf_level": self.leaf_level, "levels": n, "level_depth": list(self.level_depth[:n]),
                "L": list(self.L[:n]), "n_point_clusters": list(self.n_point_clusters[:n]),
                "n_interactions": list(self.n_interactions[:n]), "n_offsets": list(self.n_offsets[:n]),
                "near_pairs": self.near_pairs, "far_pairs": self.far_pairs, "n_point_leaves": self.n_point_leaves}


def field_plan_stats_host(nodes, tris, points, freq, c=343.0, params=None) -> dict:
    """The field-point plan of the FMM evaluation path, built on the host
    only (no GPU needed)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    p = params if params is not None else default_params()
    st = FieldStats()
    _check(lib().bem_field_plan_stats_host(nodes.ctypes.data_as(ctypes.c_void_p), nodes.shape[0],
                                           tris.ctypes.data_as(ctypes.c_void_p), tris.shape[0],
                                           pts.ctypes.data_as(ctypes.c_void_p), pts.shape[0], ctypes.byref(p),
                                           float(freq), float(c), ctypes.byref(st)))
    return st.as_dict()


class Mesh:
    """A surface mesh on the current CUDA device (App. A of the paper).

    nodes float64 [n_nodes, 3], tris int32 [n_tris, 3]; bc_type (VELO, PRES
    or ADMI per element), bc_value (complex per element) and region (per
    element, for admittances by region) as bem_mesh_create takes them.
    params: a Params (the C struct bem_params), or keyword overrides of its
    library defaults, e.g. Mesh(nodes, tris, trunc_factor=8.0,
    block_jacobi=1, near_transpose=0); every field is described in
    include/bemfmm.h."""

    def __init__(self, nodes, tris, bc_type=None, bc_value=None, region=None, params=None, **kw):
        L = lib()
        self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        self._tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.n = self._tris.shape[0]
        bt = None if bc_type is None else np.ascontiguousarray(bc_type, dtype=np.int32)
        bv = None
        if bc_value is not None:
            v = np.asarray(bc_value, dtype=np.complex128).reshape(-1)
            bv = np.ascontiguousarray(np.stack([v.real, v.imag], axis=1))
        rg = None if region is None else np.ascontiguousarray(region, dtype=np.int32)
        p = params if params is not None else default_params(**kw)
        self.params = p
        h = ctypes.c_void_p()
        ptr = (lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p))
        _check(L.bem_mesh_create(ptr(self._nodes), self._nodes.shape[0], ptr(self._tris), self.n, ptr(bt), ptr(bv),
                                 ptr(rg), ctypes.byref(p), ctypes.byref(h)), allow_warn=False)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().bem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _medium(c, rho):
        return Medium(float(c), float(rho))

    def matvec(self, freq, x, y=None, admittance=None, c=343.0, rho=1.21, stream=None):
        """y = A x (Eq. SystemI in the unknowns u); x: complex64 CUDA tensor
        [n] or [n_rhs, n] in the caller's element order."""
        import torch
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = torch.empty_like(x)
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        code = lib().bem_matvec(self._h, float(freq), ctypes.byref(med),
                                None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg,
                                _dptr(x, nrhs * self.n), _dptr(y, nrhs * self.n), nrhs, _stream_ptr(stream))
        _check(code)
        return y

    def matvec_transpose(self, freq, x, y=None, admittance=None, c=343.0, rho=1.21, stream=None):
        """y = A^T x (the adjoint solve's product); x: complex64 CUDA tensor
        [n] in the caller's element order."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        _check(lib().bem_matvec_transpose(self._h, float(freq), ctypes.byref(med),
                                          None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg,
                                          _dptr(x, self.n), _dptr(y, self.n), _stream_ptr(stream)))
        return y

    def matvec_host(self, freq, x, admittance=None, c=343.0, rho=1.21):
        """As matvec with host arrays (copies inside the call)."""
        xh = np.ascontiguousarray(np.asarray(x, dtype=np.complex64))
        yh = np.empty_like(xh)
        nrhs = 1 if xh.ndim == 1 else xh.shape[0]
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        _check(lib().bem_matvec_host(self._h, float(freq), ctypes.byref(med),
                                     None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg,
                                     xh.ctypes.data_as(ctypes.c_void_p), yh.ctypes.data_as(ctypes.c_void_p), nrhs,
                                     None))
        return yh

    def solve(self, freq, sources=(), admittance=None, tol=1e-6, max_iter=1000, c=343.0, rho=1.21, p=None, q=None,
              stream=None):
        """Solve Eq. SystemI; returns (p, q, info) as complex64 CUDA tensors
        in the caller's element order."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if p is None:
            p = torch.empty(self.n, dtype=torch.complex64, device=dev)
        if q is None:
            q = torch.empty(self.n, dtype=torch.complex64, device=dev)
        srcs = (Source * max(1, len(sources)))(*sources)
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        info = SolveInfo()
        code = lib().bem_solve(self._h, float(freq), ctypes.byref(med),
                               None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg, srcs,
                               len(sources), float(tol), int(max_iter), _dptr(p, self.n), _dptr(q, self.n),
                               ctypes.byref(info), _stream_ptr(stream))
        _check(code)
        d = {"iterations": info.iterations, "restarts": info.restarts, "relres": info.relres,
             "seconds": info.seconds, "levels": info.levels, "L": list(info.L[:info.levels]),
             "near_nnz": info.near_nnz, "status": code, "converged": code != W_NOT_CONVERGED,
             "setup_seconds": info.setup_seconds, "rhs_seconds": info.rhs_seconds,
             "gmres_seconds": info.gmres_seconds}
        return p, q, d

    def solve_multi(self, freq, sources, admittance=None, tol=1e-6, max_iter=1000, c=343.0, rho=1.21, p=None,
                    q=None, stream=None):
        """One system per source (1..4 of them), solved together (see
        bem_solve_multi); returns (p, q, infos) with p, q complex64 CUDA
        tensors [n_rhs, n_tris] in the caller's element order."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        nr = len(sources)
        if p is None:
            p = torch.empty((nr, self.n), dtype=torch.complex64, device=dev)
        if q is None:
            q = torch.empty((nr, self.n), dtype=torch.complex64, device=dev)
        srcs = (Source * nr)(*sources)
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        infos = (SolveInfo * nr)()
        code = lib().bem_solve_multi(self._h, float(freq), ctypes.byref(med),
                                     None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg, srcs, nr,
                                     float(tol), int(max_iter), _dptr(p, nr * self.n), _dptr(q, nr * self.n), infos,
                                     _stream_ptr(stream))
        _check(code)
        out = []
        for info in infos:
            out.append({"iterations": info.iterations, "restarts": info.restarts, "relres": info.relres,
                        "status": info.status, "converged": info.status != W_NOT_CONVERGED,
                        "seconds": info.seconds, "gmres_seconds": info.gmres_seconds})
        return p, q, out

    def solve_sweep(self, freqs, sources=(), admittance=None, tol=1e-6, max_iter=1000, c=343.0, rho=1.21,
                    points=None, p=None, q=None, field=None, stream=None):
        """Solve Eq. SystemI at each frequency of freqs (the next frequency's
        plan and near-field entries are prepared while the current one is
        solved); returns (p, q, field, infos): complex64 CUDA tensors
        [n_freq, n_tris] (field [n_freq, n_points], or None without points)
        and one info dict per frequency."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        fr = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).reshape(-1))
        nf = fr.shape[0]
        if p is None:
            p = torch.empty((nf, self.n), dtype=torch.complex64, device=dev)
        if q is None:
            q = torch.empty((nf, self.n), dtype=torch.complex64, device=dev)
        npts = 0
        pts = None
        if points is not None:
            pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
            npts = pts.shape[0]
            if field is None:
                field = torch.empty((nf, npts), dtype=torch.complex64, device=dev)
        srcs = (Source * max(1, len(sources)))(*sources)
        adm, nreg = _admittance(admittance)
        med = self._medium(c, rho)
        infos = (SolveInfo * nf)()
        code = lib().bem_solve_sweep(self._h, fr.ctypes.data_as(ctypes.c_void_p), nf, ctypes.byref(med),
                                     None if adm is None else adm.ctypes.data_as(ctypes.c_void_p), nreg, srcs,
                                     len(sources), float(tol), int(max_iter), _dptr(p, nf * self.n),
                                     _dptr(q, nf * self.n),
                                     None if pts is None else pts.ctypes.data_as(ctypes.c_void_p), npts,
                                     None if field is None else _dptr(field, nf * npts), infos,
                                     _stream_ptr(stream))
        _check(code)
        out = []
        for info in infos:
            out.append({"iterations": info.iterations, "restarts": info.restarts, "relres": info.relres,
                        "seconds": info.seconds, "levels": info.levels, "L": list(info.L[:info.levels]),
                        "near_nnz": info.near_nnz, "status": info.status,
                        "converged": info.status != W_NOT_CONVERGED, "setup_seconds": info.setup_seconds,
                        "rhs_seconds": info.rhs_seconds, "gmres_seconds": info.gmres_seconds})
        return p, q, (field if npts else None), out

    def evaluate(self, freq, p, q, points, sources=(), c=343.0, rho=1.21, out=None, stream=None):
        """Total pressure at exterior points (Eq. BIE_I, lambda = 1)."""
        import torch
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
        m = pts.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.complex64, device=p.device)
        srcs = (Source * max(1, len(sources)))(*sources)
        med = self._medium(c, rho)
        _check(lib().bem_evaluate(self._h, float(freq), ctypes.byref(med), srcs, len(sources), _dptr(p, self.n),
                                  _dptr(q, self.n), pts.ctypes.data_as(ctypes.c_void_p), m, _dptr(out, m),
                                  _stream_ptr(stream)))
        return out

    def evaluate_velocity(self, freq, p, q, points, sources=(), c=343.0, rho=1.21, out=None, stream=None):
        """Particle velocity v = grad p / (i w rho) at exterior points
        (Eq. utopandv with Eq. BIE_I differentiated); complex64 [M, 3]."""
        import torch
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
        m = pts.shape[0]
        if out is None:
            out = torch.empty((m, 3), dtype=torch.complex64, device=p.device)
        srcs = (Source * max(1, len(sources)))(*sources)
        med = self._medium(c, rho)
        _check(lib().bem_evaluate_velocity(self._h, float(freq), ctypes.byref(med), srcs, len(sources),
                                           _dptr(p, self.n), _dptr(q, self.n), pts.ctypes.data_as(ctypes.c_void_p),
                                           m, _dptr(out, 3 * m), _stream_ptr(stream)))
        return out

    def admittance_gradient(self, freq, sources, admittance, points, tol=1e-7, max_iter=1000, c=343.0, rho=1.21,
                            p=None, q=None, stream=None):
        """Loss L = sum_m |p(x_m)|^2 of the total pressure at the points and
        its gradient dL/dRe Y_r + i dL/dIm Y_r with respect to the region
        admittances, by the adjoint of Eq. SystemI.
        Returns (L, grad complex128 [n_regions], p, q, info), p and q the
        forward solution (complex64 CUDA tensors, caller order)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if p is None:
            p = torch.empty(self.n, dtype=torch.complex64, device=dev)
        if q is None:
            q = torch.empty(self.n, dtype=torch.complex64, device=dev)
        adm, nreg = _admittance(admittance)
        if adm is None:
            raise ValueError("admittance per region is required")
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
        srcs = (Source * max(1, len(sources)))(*sources)
        med = self._medium(c, rho)
        info = SolveInfo()
        loss = ctypes.c_double(0.0)
        grad = np.zeros(2 * nreg, dtype=np.float64)
        code = lib().bem_admittance_gradient(self._h, float(freq), ctypes.byref(med),
                                             adm.ctypes.data_as(ctypes.c_void_p), nreg, srcs, len(sources),
                                             pts.ctypes.data_as(ctypes.c_void_p), pts.shape[0], float(tol),
                                             int(max_iter), _dptr(p, self.n), _dptr(q, self.n), ctypes.byref(loss),
                                             grad.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info),
                                             _stream_ptr(stream))
        _check(code)
        d = {"iterations": info.iterations, "restarts": info.restarts, "relres": info.relres,
             "status": code, "converged": code != W_NOT_CONVERGED}
        return loss.value, grad[0::2] + 1j * grad[1::2], p, q, d

    def blocks(self, freq, c=343.0, rho=1.21):
        """Sub-block index of each element (caller order) of the block-Jacobi
        preconditioner in the plan for freq (int32 numpy array [n])."""
        out = np.empty(self.n, dtype=np.int32)
        med = self._medium(c, rho)
        _check(lib().bem_mesh_blocks(self._h, float(freq), ctypes.byref(med), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def krylov_basis(self, plane=0, max_cols=1024):
        """The last GMRES cycle's basis vectors as a [cols, n] complex64 device
        tensor (internal element order)."""
        import torch
        v = torch.empty((max_cols, self.n), dtype=torch.complex64, device="cuda")
        nc = ctypes.c_int32(0)
        _check(lib().bem_krylov_basis(self._h, int(plane), _dptr(v, max_cols * self.n), int(max_cols),
                                      ctypes.byref(nc)))
        return v[:min(nc.value, max_cols)]

    def release_plan(self):
        """Free the per-frequency plan; the next call rebuilds it."""
        _check(lib().bem_mesh_release_plan(self._h))

    def stats(self, freq, c=343.0, rho=1.21) -> dict:
        st = PlanStats()
        med = self._medium(c, rho)
        _check(lib().bem_mesh_stats(self._h, float(freq), ctypes.byref(med), ctypes.byref(st)))
        return st.as_dict()


def _admittance_loss_fn():
    import torch

    class AdmittanceLoss(torch.autograd.Function):
        """L(Y) = sum_m |p(x_m)|^2 as a differentiable function of the region
        admittances Y (complex tensor [n_regions]); the backward pass returns
        the adjoint gradient bem_admittance_gradient computed with the
        forward one (PyTorch's convention for a real function of complex
        inputs: dL/dRe Y + i dL/dIm Y)."""

        @staticmethod
        def forward(ctx, Y, mesh, freq, sources, points, tol, c, rho):
            y = Y.detach().cpu().numpy().astype(np.complex128)
            L, g, _, _, info = mesh.admittance_gradient(freq, sources, y, points, tol=tol, c=c, rho=rho)
            if not info["converged"]:
                raise BemError(W_NOT_CONVERGED, lib().bem_last_error().decode(errors="replace"))
            ctx.save_for_backward(torch.as_tensor(g, dtype=Y.dtype, device=Y.device))
            return torch.as_tensor(L, dtype=Y.real.dtype, device=Y.device)

        @staticmethod
        def backward(ctx, gL):
            (g,) = ctx.saved_tensors
            return gL * g, None, None, None, None, None, None, None

    return AdmittanceLoss


def admittance_loss(mesh, Y, freq, sources, points, tol=1e-7, c=343.0, rho=1.21):
    """Differentiable field loss sum_m |p(x_m)|^2 of the region admittances
    Y (complex torch tensor [n_regions], e.g. with requires_grad); see
    Mesh.admittance_gradient."""
    global _AdmittanceLoss
    if _AdmittanceLoss is None:
        _AdmittanceLoss = _admittance_loss_fn()
    return _AdmittanceLoss.apply(Y, mesh, float(freq), tuple(sources), points, float(tol), float(c), float(rho))


_AdmittanceLoss = None
