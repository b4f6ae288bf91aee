"""Closed-form solutions used to pin the oracle (independent of it).

Time factor e^{-iwt}, outgoing h_n = h_n^{(1)} (consistent with
G = e^{ikr}/(4 pi r) of Eq. BIE_I).  Spherical Bessel functions come from
scipy.special (a library primitive).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def _h(n, x, derivative=False):
    return spherical_jn(n, x, derivative) + 1j * spherical_yn(n, x, derivative)


def sphere_plane_wave(points, k, a, beta=0.0, nmax=None):
    """Total pressure for a unit plane wave e^{ikz} scattered by a sphere of
    radius a centred at the origin, with the wall condition dp/dr = -i k beta p
    at r = a (beta = rho c Y; beta = 0 is sound hard).  Points with r < a are
    evaluated at r = a (surface value at the point's polar angle).

    p = sum_n i^n (2n+1) [j_n(kr) + b_n h_n(kr)] P_n(cos theta),
    b_n = -(j_n'(ka) + i beta j_n(ka)) / (h_n'(ka) + i beta h_n(ka))."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 2] / r
    rr = np.maximum(r, a)
    ka = k * a
    if nmax is None:
        nmax = int(ka + 30 + 2 * np.max(k * rr))
    p = np.zeros(pts.shape[0], np.complex128)
    on_surface = r <= a * (1 + 1e-12)
    for n in range(nmax + 1):
        jn_a, djn_a = spherical_jn(n, ka), spherical_jn(n, ka, True)
        hn_a, dhn_a = _h(n, ka), _h(n, ka, True)
        bn = -(djn_a + 1j * beta * jn_a) / (dhn_a + 1j * beta * hn_a)
        Pn = eval_legendre(n, ct)
        coef = (1j ** n) * (2 * n + 1)
        radial = spherical_jn(n, k * rr) + bn * _h(n, k * rr)
        if beta == 0.0:
            # on the surface use the Wronskian form (exact cancellation)
            surf = 1j / (ka * ka) / dhn_a
            radial = np.where(on_surface, surf, radial)
        p += coef * radial * Pn
    return p


def sphere_plane_wave_dbeta(points, k, a, beta, nmax=None):
    """Derivative dp/d(beta) of the exterior field of sphere_plane_wave (points
    with r > a).  Only b_n depends on beta; by the quotient rule
    db_n/dbeta = -i [j_n (h_n' + i beta h_n) - h_n (j_n' + i beta j_n)]
                 / (h_n' + i beta h_n)^2   (Bessel values at ka)."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(pts, axis=1)
    if np.any(r <= a):
        raise ValueError("exterior points only")
    ct = pts[:, 2] / r
    ka = k * a
    if nmax is None:
        nmax = int(ka + 30 + 2 * np.max(k * r))
    dp = np.zeros(pts.shape[0], np.complex128)
    for n in range(nmax + 1):
        jn_a, djn_a = spherical_jn(n, ka), spherical_jn(n, ka, True)
        hn_a, dhn_a = _h(n, ka), _h(n, ka, True)
        den = dhn_a + 1j * beta * hn_a
        dbn = -1j * (jn_a * den - hn_a * (djn_a + 1j * beta * jn_a)) / (den * den)
        dp += (1j ** n) * (2 * n + 1) * dbn * _h(n, k * r) * eval_legendre(n, ct)
    return dp


def monopole(points, x0, k, amp=1.0):
    """Free-field point source amp e^{ikR}/(4 pi R) and its gradient."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    d = pts - np.asarray(x0, dtype=np.float64)[None, :]
    R = np.linalg.norm(d, axis=1)
    G = amp * np.exp(1j * k * R) / (4 * np.pi * R)
    grad = (G * (1j * k - 1.0 / R) / R)[:, None] * d
    return G, grad


def disk_G(k, R):
    """Integral of e^{ikr}/(4 pi r) over a disk of radius R about its centre."""
    return (np.exp(1j * k * R) - 1.0) / (2j * k) if k != 0 else R / 2.0


def disk_E(k, R):
    """Hadamard finite part of the integral of d2G/dn_x dn_y over a planar disk
    of radius R about its centre: (ik - e^{ikR}/R) / 2."""
    return 0.5 * (1j * k - np.exp(1j * k * R) / R)


def polygon_static_G(x, poly):
    """Integral of 1/(4 pi r) over a planar polygon from a point x in its plane
    and inside it: (1/4 pi) sum_e d_e ln[(s+ + R+)/(s- + R-)]."""
    poly = np.asarray(poly, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    tot = 0.0
    nv = poly.shape[0]
    for e in range(nv):
        P, Q = poly[e], poly[(e + 1) % nv]
        t = (Q - P) / np.linalg.norm(Q - P)
        foot = P + np.dot(x - P, t) * t
        d = np.linalg.norm(x - foot)
        sm, sp = np.dot(P - foot, t), np.dot(Q - foot, t)
        Rm, Rp = np.linalg.norm(P - x), np.linalg.norm(Q - x)
        tot += d * np.log((sp + Rp) / (sm + Rm))
    return tot / (4 * np.pi)


def polygon_static_E(x, poly):
    """Hadamard finite part of the integral of E = d2G/dn_x dn_y at k = 0
    (E = 1/(4 pi r^3) for points in the plane) over a planar polygon that
    contains x:  -(1/4 pi) sum_e (1/d_e) [s / sqrt(d_e^2 + s^2)]_{s-}^{s+}."""
    poly = np.asarray(poly, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    tot = 0.0
    nv = poly.shape[0]
    for e in range(nv):
        P, Q = poly[e], poly[(e + 1) % nv]
        t = (Q - P) / np.linalg.norm(Q - P)
        foot = P + np.dot(x - P, t) * t
        d = np.linalg.norm(x - foot)
        sm, sp = np.dot(P - foot, t), np.dot(Q - foot, t)
        tot += (sp / np.hypot(d, sp) - sm / np.hypot(d, sm)) / d
    return -tot / (4 * np.pi)


def sph_hankel_closed(n, x):
    """h_n^{(1)}(x) for n <= 3 from the elementary closed forms."""
    e = np.exp(1j * x)
    if n == 0:
        return -1j * e / x
    if n == 1:
        return -e * (x + 1j) / x ** 2
    if n == 2:
        return 1j * e * (x * x + 3j * x - 3) / x ** 3
    if n == 3:
        return e * (x ** 3 + 6j * x * x - 15 * x - 15j) / x ** 4
    raise ValueError(n)
