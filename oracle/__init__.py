"""Plain CPU FP64 oracle for the collocation BEM of arXiv 2312.00005.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library package
never does.  The arithmetic lives in ``bem_oracle.c`` (plain C, FP64, OpenMP
over rows); this file compiles it with gcc on first use and wraps it with
ctypes, and states the boundary-condition bookkeeping of Eq. SystemI in
pressure variables.

Conventions (pressure form, exterior problem tau = 1, time factor e^{-iwt}):
  q = dp/dn = i w rho v  (Eq. utopandv, v the normal particle velocity);
  boundary types: VELO (v given; default v = 0 is sound hard), PRES (p given),
  ADMI (admittance Y: velocity into the wall = Y p, i.e. q = -i k beta p with
  beta = rho c Y, plus an optional extra velocity);
  Burton-Miller: gamma = i/k (Eq. SystemI).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "lib", "build", "VELO", "PRES", "ADMI", "geometry", "gauss_legendre", "gauss_jacobi10",
    "triangle_rule", "quad_order", "kernels", "element_integrals", "duffy_G", "edge_fp",
    "column_coeffs", "assemble", "matvec_rows", "matvec_dense", "gmres", "incident", "rhs",
    "solve", "field", "field_velocity", "field_matrices", "admittance_gradient", "sph_hankel", "sphere_grid", "translation", "fmm_pair", "num_threads",
    "OracleError",
]

VELO, PRES, ADMI = 0, 1, 2
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_SO = os.path.join(_HERE, "_bem_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    """Raised when the oracle reports the subdivision-limit error (Sec. 4.1)."""

    def __init__(self, msg, element=-1):
        super().__init__(msg)
        self.element = element


def build(force: bool = False) -> str:
    """Compile bem_oracle.c into _bem_oracle.so with gcc (plain C11, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
            P = ctypes.c_void_p
            sig = {
                "orc_gauss_legendre": (i, [i, P, P]),
                "orc_gauss_jacobi10": (i, [i, P, P]),
                "orc_triangle_rule": (i, [i, P, P, P]),
                "orc_quad_order": (i, [d, d, i]),
                "orc_kernels": (None, [P, P, P, P, d, P]),
                "orc_duffy_G": (None, [P, P, i, d, i, P]),
                "orc_edge_fp": (None, [P, P, P, i, d, i, i, P]),
                "orc_element_integrals": (i, [P, P, P, P, P, i, d, P, P]),
                "orc_geometry": (None, [P, P, l, P, P, P]),
                "orc_assemble": (i, [P, P, l, d, P, P, P, P, P]),
                "orc_matvec_rows": (i, [P, P, l, d, P, P, P, P, P, l, P, P]),
                "orc_matvec_dense": (None, [P, l, P, P]),
                "orc_matvec_block": (None, [P, l, l, P, P]),
                "orc_gmres": (i, [P, l, P, P, d, i, i, P, P]),
                "orc_incident": (None, [P, P, l, d, i, P, P, P, P]),
                "orc_field": (i, [P, P, l, d, P, P, P, P, l, P, P]),
                "orc_field_grad": (i, [P, P, l, d, P, P, P, P, l, P, P]),
                "orc_field_mats": (i, [P, P, l, d, P, P, l, P, P, P]),
                "orc_sph_hankel": (None, [i, d, P]),
                "orc_sphere_grid": (i, [i, P, P]),
                "orc_translation": (None, [i, d, P, P, i, P]),
                "orc_fmm_pair": (i, [P, P, P, P, d, i, P]),
                "orc_num_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _params(params):
    if params is None:
        return None
    keys = ["quad_tol", "m_max", "rt_subdiv", "max_depth", "n_duffy", "edge_parts", "edge_gauss", "tau"]
    dflt = {"quad_tol": 1e-3, "m_max": 6, "rt_subdiv": 1.3, "max_depth": 15, "n_duffy": 4,
            "edge_parts": 4, "edge_gauss": 3, "tau": 1.0}
    dflt.update(params)
    return np.array([float(dflt[k]) for k in keys], dtype=np.float64)


def _pp(arr):
    return None if arr is None else _p(arr)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- rules
def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    if lib().orc_gauss_legendre(n, _p(x), _p(w)):
        raise RuntimeError("gauss_legendre failed")
    return x, w


def gauss_jacobi10(n):
    x, w = np.zeros(n), np.zeros(n)
    if lib().orc_gauss_jacobi10(n, _p(x), _p(w)):
        raise RuntimeError("gauss_jacobi10 failed")
    return x, w


def triangle_rule(m):
    xi, eta, w = np.zeros(m * m), np.zeros(m * m), np.zeros(m * m)
    if lib().orc_triangle_rule(m, _p(xi), _p(eta), _p(w)):
        raise RuntimeError("triangle_rule failed")
    return xi, eta, w


def quad_order(rt, tol=1e-3, m_max=6):
    return int(lib().orc_quad_order(float(rt), float(tol), int(m_max)))


# ---------------------------------------------------------------- kernels / integrals
def kernels(x, nx, y, ny, k):
    """(G, H, H', E) at one pair of points."""
    out = np.zeros(8)
    lib().orc_kernels(_p(_f64(x)), _p(_f64(nx)), _p(_f64(y)), _p(_f64(ny)), float(k), _p(out))
    return out.view(np.complex128)


def element_integrals(x, nx, a, b, c, k, self_term=False, params=None):
    """Integrals of (G, H, H', E) over triangle (a, b, c) at point x."""
    out = np.zeros(8)
    pr = _params(params)
    st = lib().orc_element_integrals(_p(_f64(x)), _p(_f64(nx)), _p(_f64(a)), _p(_f64(b)),
                                     _p(_f64(c)), int(bool(self_term)), float(k), _pp(pr), _p(out))
    if st:
        raise OracleError("subdivision limit exceeded")
    return out.view(np.complex128)


def duffy_G(x, poly, k, n=4):
    out = np.zeros(2)
    poly = _f64(poly, (-1, 3))
    lib().orc_duffy_G(_p(_f64(x)), _p(poly), poly.shape[0], float(k), int(n), _p(out))
    return complex(out[0], out[1])


def edge_fp(x, normal, poly, k, parts=4, ng=3):
    out = np.zeros(2)
    poly = _f64(poly, (-1, 3))
    lib().orc_edge_fp(_p(_f64(x)), _p(_f64(normal)), _p(poly), poly.shape[0], float(k), int(parts),
                      int(ng), _p(out))
    return complex(out[0], out[1])


def geometry(nodes, tris):
    """(midpoints [N,3], unit normals [N,3], areas [N])."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    cen, nrm, area = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().orc_geometry(_p(nodes), _p(tris), n, _p(cen), _p(nrm), _p(area))
    return cen, nrm, area


# ---------------------------------------------------------------- system
def column_coeffs(bc_type, k, c, rho, beta=None, tau=1.0):
    """Column coefficients (cp, cq) of the unknown vector and (cp0, cq0) of the
    known-data vector (Eq. SystemI, pressure form).

    beta = rho c Y per element (only used on ADMI elements), Y the velocity
    into the wall over p: along the normal for the interior problem
    (tau = -1, normals out of the fluid), against it for the exterior
    problem, so q = dp/dn = -tau i k beta p."""
    bc_type = np.asarray(bc_type)
    n = bc_type.shape[0]
    cp = np.zeros(n, np.complex128)
    cq = np.zeros(n, np.complex128)
    cp0 = np.zeros(n, np.complex128)
    cq0 = np.zeros(n, np.complex128)
    pu = bc_type != PRES
    cp[pu] = 1.0
    adm = bc_type == ADMI
    if adm.any():
        cq[adm] = -1j * k * tau * np.asarray(beta)[adm]
    cq[~pu] = 1.0
    cq0[pu] = 1.0          # known q-part g on VELO / ADMI elements
    cp0[~pu] = 1.0         # known p on PRES elements
    return cp, cq, cp0, cq0


def known_data(bc_type, bc_value, omega, rho):
    """Known vector: g = i w rho v on VELO / ADMI elements, p on PRES."""
    bc_type = np.asarray(bc_type)
    v = _c128(bc_value)
    z = np.where(bc_type == PRES, v, 1j * omega * rho * v)
    return z.astype(np.complex128)


def assemble(nodes, tris, k, cp, cq, params=None):
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    A = np.zeros((n, n), np.complex128)
    bad = ctypes.c_long(-1)
    cp, cq = _c128(cp), _c128(cq)
    pr = _params(params)
    st = lib().orc_assemble(_p(nodes), _p(tris), n, float(k), _p(cp), _p(cq), _pp(pr), _p(A),
                            ctypes.byref(bad))
    if st:
        raise OracleError("number of subdivisions exceeds the limit at element %d" % bad.value,
                          bad.value)
    return A


def matvec_rows(nodes, tris, k, cp, cq, x, rows, params=None):
    """(A x)[rows] with the entries computed on the fly (no N x N storage)."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    y = np.zeros(rows.shape[0], np.complex128)
    bad = ctypes.c_long(-1)
    cp, cq, x = _c128(cp), _c128(cq), _c128(x)
    pr = _params(params)
    st = lib().orc_matvec_rows(_p(nodes), _p(tris), n, float(k), _p(cp), _p(cq), _pp(pr), _p(x),
                               _p(rows), rows.shape[0], _p(y), ctypes.byref(bad))
    if st:
        raise OracleError("number of subdivisions exceeds the limit at element %d" % bad.value,
                          bad.value)
    return y


def matvec_dense(A, x):
    A, x = _c128(A), _c128(x)
    y = np.zeros(A.shape[0], np.complex128)
    lib().orc_matvec_dense(_p(A), A.shape[0], _p(x), _p(y))
    return y


def matvec_dense_block(A, x):
    """y = A x for a dense (rows x n) block."""
    A, x = _c128(A), _c128(x)
    y = np.zeros(A.shape[0], np.complex128)
    lib().orc_matvec_block(_p(A), A.shape[0], A.shape[1], _p(x), _p(y))
    return y


def gmres(A, b, tol=1e-8, maxit=1000, restart=200):
    A, b = _c128(A), _c128(b)
    x = np.zeros(b.shape[0], np.complex128)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    st = lib().orc_gmres(_p(A), A.shape[0], _p(b), _p(x), float(tol), int(maxit), int(restart),
                         ctypes.byref(it), ctypes.byref(rr))
    return x, {"converged": st == 0, "iterations": it.value, "relres": rr.value}


def incident(x, nx, k, kind, vec, amp=1.0 + 0.0j):
    """Incident pressure p and dp/dn at points x (normals nx or None).
    kind 'plane' (vec = direction) or 'point' (vec = source position)."""
    x = _f64(x, (-1, 3))
    m = x.shape[0]
    p = np.zeros(m, np.complex128)
    dp = np.zeros(m, np.complex128)
    a = np.array([complex(amp).real, complex(amp).imag])
    nxa = None if nx is None else _f64(nx, (-1, 3))
    lib().orc_incident(_p(x), _pp(nxa), m, float(k), 0 if kind == "plane" else 1, _p(_f64(vec)),
                       _p(a), _p(p), _p(dp))
    return p, (dp if nx is not None else None)


def rhs(cen, nrm, k, sources):
    """b_inc = p_inc - gamma dp_inc/dn at the collocation points (Eq. SystemI)."""
    gamma = 1j / k
    b = np.zeros(cen.shape[0], np.complex128)
    for (kind, vec, amp) in sources:
        p, dp = incident(cen, nrm, k, kind, vec, amp)
        b += p - gamma * dp
    return b


def solve(nodes, tris, freq, c=343.0, rho=1.21, sources=(), bc_type=None, bc_value=None,
          beta=None, tol=1e-8, maxit=2000, restart=300, params=None, return_system=False,
          row_scaling=False, blocks=None):
    """Dense collocation BEM solve (Eq. SystemI) with GMRES.

    sources: iterable of (kind, vector, complex amplitude).
    bc_type / bc_value: per element (default all VELO with v = 0).
    beta: per-element rho c Y for ADMI elements.
    row_scaling: GMRES on D^-1 A u = D^-1 b with D = diag(A), the solver's
    row-scaling preconditioner (Sec. 3.2); tol then applies to the scaled
    residual.
    blocks: per element a block index; GMRES on P A u = P b with P the
    inverse of A's block diagonal over those blocks (block-Jacobi, the block
    form of row scaling; singleton blocks are row scaling).
    Returns (p, q, info) at the element midpoints."""
    tris = _i32(tris)
    n = tris.shape[0]
    k = 2.0 * np.pi * freq / c
    omega = 2.0 * np.pi * freq
    bc_type = np.zeros(n, np.int32) if bc_type is None else np.asarray(bc_type, np.int32)
    bc_value = np.zeros(n, np.complex128) if bc_value is None else _c128(bc_value)
    tau = -1.0 if params is not None and params.get("tau", 1.0) < 0 else 1.0
    cp, cq, cp0, cq0 = column_coeffs(bc_type, k, c, rho, beta, tau)
    cen, nrm, _ = geometry(nodes, tris)
    b = rhs(cen, nrm, k, sources)
    z = known_data(bc_type, bc_value, omega, rho)
    if np.any(z != 0):
        A0 = assemble(nodes, tris, k, cp0, cq0, params)
        b = b - A0 @ z
        del A0
    A = assemble(nodes, tris, k, cp, cq, params)
    if row_scaling:
        dinv = 1.0 / np.diag(A)
        u, info = gmres(A * dinv[:, None], b * dinv, tol=tol, maxit=maxit, restart=restart)
    elif blocks is not None:
        blocks = np.asarray(blocks)
        PA, Pb = np.empty_like(A), np.empty_like(b)
        for c in np.unique(blocks):
            idx = np.where(blocks == c)[0]
            lu = np.linalg.inv(A[np.ix_(idx, idx)])
            PA[idx] = lu @ A[idx]
            Pb[idx] = lu @ b[idx]
        u, info = gmres(PA, Pb, tol=tol, maxit=maxit, restart=restart)
    else:
        u, info = gmres(A, b, tol=tol, maxit=maxit, restart=restart)
    pu = bc_type != PRES
    p = np.where(pu, u, z)
    # on VELO / ADMI elements q = a u + g (cq holds a = -ik beta, zero for VELO)
    q = np.where(pu, np.where(bc_type == ADMI, cq, 0.0) * u + z, u)
    if return_system:
        return p, q, info, (A, b)
    return p, q, info


def field(nodes, tris, freq, p, q, pts, c=343.0, sources=(), params=None):
    """Total pressure at exterior points: p_inc + sum_j [H_j p_j - G_j q_j]
    (Eq. BIE_I with lambda = 1, tau = 1)."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    pts = _f64(pts, (-1, 3))
    k = 2.0 * np.pi * freq / c
    out = np.zeros(pts.shape[0], np.complex128)
    bad = ctypes.c_long(-1)
    pr = _params(params)
    st = lib().orc_field(_p(nodes), _p(tris), n, float(k), _p(_c128(p)), _p(_c128(q)), _pp(pr),
                         _p(pts), pts.shape[0], _p(out), ctypes.byref(bad))
    if st:
        raise OracleError("number of subdivisions exceeds the limit at element %d" % bad.value,
                          bad.value)
    for (kind, vec, amp) in sources:
        pi, _ = incident(pts, None, k, kind, vec, amp)
        out += pi
    return out


def field_velocity(nodes, tris, freq, p, q, pts, c=343.0, rho=1.21, sources=(), params=None):
    """Particle velocity at exterior points, v = grad p / (i w rho)
    (Eq. utopandv), with grad p = grad p_inc + sum_j [grad H_j p_j - grad G_j q_j]
    (Eq. BIE_I, lambda = 1, differentiated under the integral; the component
    along an axis e uses the kernels H' and E of Eq. dBIE with n_x = e).
    Returns complex [npts, 3]."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    pts = _f64(pts, (-1, 3))
    k = 2.0 * np.pi * freq / c
    grad = np.zeros((pts.shape[0], 3), np.complex128)
    bad = ctypes.c_long(-1)
    pr = _params(params)
    st = lib().orc_field_grad(_p(nodes), _p(tris), n, float(k), _p(_c128(p)), _p(_c128(q)), _pp(pr),
                              _p(pts), pts.shape[0], _p(grad), ctypes.byref(bad))
    if st:
        raise OracleError("number of subdivisions exceeds the limit at element %d" % bad.value,
                          bad.value)
    for (kind, vec, amp) in sources:
        for ax in range(3):
            e = np.zeros_like(pts)
            e[:, ax] = 1.0
            _, dpi = incident(pts, e, k, kind, vec, amp)
            grad[:, ax] += dpi
    omega = 2.0 * np.pi * freq
    return grad / (1j * omega * rho)


def field_matrices(nodes, tris, freq, pts, c=343.0, params=None):
    """(Gm, Hm): the element integrals G(x_r)_j and H(x_r)_j of the
    representation formula (Eq. BIE_I, lambda = 1) as dense [npts, N]
    matrices, without the tau sign (the field is p_inc + tau (Hm p - Gm q))."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    pts = _f64(pts, (-1, 3))
    k = 2.0 * np.pi * freq / c
    Gm = np.zeros((pts.shape[0], n), np.complex128)
    Hm = np.zeros((pts.shape[0], n), np.complex128)
    bad = ctypes.c_long(-1)
    st = lib().orc_field_mats(_p(nodes), _p(tris), n, float(k), _pp(_params(params)), _p(pts), pts.shape[0],
                              _p(Gm), _p(Hm), ctypes.byref(bad))
    if st:
        raise OracleError("number of subdivisions exceeds the limit at element %d" % bad.value,
                          bad.value)
    return Gm, Hm


def admittance_gradient(nodes, tris, freq, pts, region, Y, sources=(), bc_type=None, bc_value=None,
                        c=343.0, rho=1.21, params=None, tol=1e-12):
    """Field loss L = sum_m |p(x_m)|^2 at the points x_m and its gradient with
    respect to the region admittances Y_r, by the adjoint of the discrete
    system (a derived quantity: the paper solves the forward problem only).

    region: per element, the admittance region (index into Y) or -1; an
    element with region >= 0 is ADMI (bc_type may also be given), with
    beta_j = rho c Y_region(j) and the column coefficient
    cq_j = -tau i k beta_j of the admittance condition.
    Returns (L, grad, info) with grad_r = dL/d(Re Y_r) + i dL/d(Im Y_r).

    Steps (pressure form, Eq. SystemI and Eq. BIE_I):
      1. A is linear in the column coefficients: A = Ap diag(cp) + Aq diag(cq),
         Ap the operator on p-unknowns (cp = 1, cq = 0), Aq on q-unknowns.
      2. Forward: A u = b; p = cp u + cp0 z, q = cq u + cq0 z.
      3. Field f = p_inc + tau (Hm p - Gm q) = p_inc + F u + const with
         F = tau (Hm diag(cp) - Gm diag(cq)); L = f^H f.
      4. u and f are holomorphic in Y; with s_r = f^H df/dY_r the real
         gradient is 2 conj(s_r).
      5. df/dY_r = -tau Gm (d_r o u) - F A^-1 Aq (d_r o u), d_r = dcq/dY_r
         = -tau i k rho c on ADMI elements of region r, 0 elsewhere.
      6. Adjoint: A^T lam = F^T conj(f), so that f^H F A^-1 = lam^T; then
         s_r = sum over elements j of region r of
               d_j u_j [ -tau (Gm^T conj f)_j - (Aq^T lam)_j ]."""
    nodes, tris = _f64(nodes), _i32(tris)
    n = tris.shape[0]
    k = 2.0 * np.pi * freq / c
    omega = 2.0 * np.pi * freq
    tau = -1.0 if params is not None and params.get("tau", 1.0) < 0 else 1.0
    region = np.asarray(region, np.int64).reshape(n)
    Y = np.asarray(Y, np.complex128).reshape(-1)
    if bc_type is None:
        bc_type = np.where(region >= 0, ADMI, VELO).astype(np.int32)
    bc_type = np.asarray(bc_type, np.int32)
    adm = bc_type == ADMI
    if np.any(region[adm] < 0) or np.any(region >= Y.shape[0]):
        raise ValueError("every ADMI element needs a region index into Y")
    bc_value = np.zeros(n, np.complex128) if bc_value is None else _c128(bc_value)
    beta = np.zeros(n, np.complex128)
    beta[adm] = rho * c * Y[region[adm]]
    cp, cq, cp0, cq0 = column_coeffs(bc_type, k, c, rho, beta, tau)
    cen, nrm, _ = geometry(nodes, tris)
    b = rhs(cen, nrm, k, sources)
    z = known_data(bc_type, bc_value, omega, rho)
    if np.any(z != 0):
        b = b - assemble(nodes, tris, k, cp0, cq0, params) @ z
    ones, zeros = np.ones(n, np.complex128), np.zeros(n, np.complex128)
    Ap = assemble(nodes, tris, k, ones, zeros, params)
    Aq = assemble(nodes, tris, k, zeros, ones, params)
    A = Ap * cp[None, :] + Aq * cq[None, :]
    del Ap
    u, info_f = gmres(A, b, tol=tol, maxit=4 * n + 100, restart=min(n, 300))
    p = cp * u + cp0 * z
    q = cq * u + cq0 * z
    Gm, Hm = field_matrices(nodes, tris, freq, pts, c, params)
    f = tau * (Hm @ p - Gm @ q)
    for (kind, vec, amp) in sources:
        pi, _ = incident(pts, None, k, kind, vec, amp)
        f = f + pi
    L = float(np.real(np.vdot(f, f)))
    F = tau * (Hm * cp[None, :] - Gm * cq[None, :])
    lam, info_a = gmres(np.ascontiguousarray(A.T), F.T @ np.conj(f), tol=tol, maxit=4 * n + 100,
                        restart=min(n, 300))
    d = np.where(adm, -tau * 1j * k * rho * c, 0.0)
    t = d * u * (-tau * (Gm.T @ np.conj(f)) - Aq.T @ lam)
    s = np.zeros(Y.shape[0], np.complex128)
    np.add.at(s, region[adm], t[adm])
    grad = 2.0 * np.conj(s)
    info = {"forward": info_f, "adjoint": info_a, "p": p, "q": q, "field": f}
    return L, grad, info


# ---------------------------------------------------------------- FMM pieces (unit tests)
def sph_hankel(nmax, x):
    out = np.zeros(2 * (nmax + 1))
    lib().orc_sph_hankel(int(nmax), float(x), _p(out))
    return out.view(np.complex128)


def sphere_grid(L):
    s, w = np.zeros((2 * L * L, 3)), np.zeros(2 * L * L)
    if lib().orc_sphere_grid(int(L), _p(s), _p(w)):
        raise RuntimeError("sphere_grid failed")
    return s, w


def translation(L, k, X, s):
    s = _f64(s, (-1, 3))
    out = np.zeros(2 * s.shape[0])
    lib().orc_translation(int(L), float(k), _p(_f64(X)), _p(s), s.shape[0], _p(out))
    return out.view(np.complex128)


def fmm_pair(x, y, z1, z2, k, L):
    out = np.zeros(2)
    if lib().orc_fmm_pair(_p(_f64(x)), _p(_f64(y)), _p(_f64(z1)), _p(_f64(z2)), float(k), int(L),
                          _p(out)):
        raise RuntimeError("fmm_pair failed")
    return complex(out[0], out[1])
