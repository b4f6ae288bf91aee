"""Pins of the oracle's quadrature and kernels against closed forms, library
routines and brute force (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import spherical_jn, spherical_yn

import oracle
from closed_forms import (disk_E, disk_G, polygon_static_E, polygon_static_G,
                          sph_hankel_closed)


# ------------------------------------------------------------------ Gauss rules
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 16, 33, 64])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = oracle.gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-13 * max(1, n / 8)
    # not exact at degree 2n (pins the number of points; the defect is
    # below rounding for large n)
    if n <= 9:
        assert abs(np.dot(w, x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_gauss_jacobi10_exact(n):
    x, w = oracle.gauss_jacobi10(n)
    for p in range(2 * n):
        # int_{-1}^{1} (1 - t) t^p dt
        exact = (0.0 if p % 2 else 2.0 / (p + 1)) - (2.0 / (p + 2) if p % 2 else 0.0)
        assert abs(np.dot(w, x ** p) - exact) < 1e-13
    if n <= 9:
        exact = 2.0 / (2 * n + 1)
        assert abs(np.dot(w, x ** (2 * n)) - exact) > 1e-12


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 10])
def test_triangle_rule_exact_on_monomials(m):
    xi, eta, w = oracle.triangle_rule(m)
    assert abs(w.sum() - 0.5) < 1e-14
    assert np.all(xi >= 0) and np.all(eta >= 0) and np.all(xi + eta <= 1)
    for a in range(2 * m):
        for b in range(2 * m - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.dot(w, xi ** a * eta ** b) - exact) < 1e-14
    # degree 2m is not integrated exactly by an m x m collapsed rule
    errs = [abs(np.dot(w, xi ** a * eta ** (2 * m - a))
                - math.factorial(a) * math.factorial(2 * m - a) / math.factorial(2 * m + 2))
            for a in range(2 * m + 1)]
    if m <= 6:
        assert max(errs) > 1e-12


def test_quad_order_monotone_and_capped():
    rts = np.linspace(1.3, 60.0, 500)
    ms = [oracle.quad_order(r) for r in rts]
    assert ms[0] == 6 and ms[-1] == 1
    assert all(a >= b for a, b in zip(ms, ms[1:]))
    assert oracle.quad_order(0.5) == 6          # capped


def order_thresholds_golden():
    """(tol, m, binding estimate, R_m) rows of tests/golden/order_thresholds.txt:
    the r~ above which order m meets all three a-priori estimates of
    Sec. 3.1.4, derived by hand there from the printed formulas."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "order_thresholds.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tol, m, est, R = line.split()
        rows.append((float(tol), int(m), est, float(R)))
    return rows


@pytest.mark.parametrize("tol,m,est,R", order_thresholds_golden())
def test_quad_order_switches_at_the_hand_derived_thresholds(tol, m, est, R):
    """Just above R_m order m suffices, just below it order m + 1 is needed.
    Each estimate binds in some row (eps_G at m = 1, eps_H at m = 2, eps_E at
    m = 3..5 for tol 1e-3; eps_G at m = 2 and eps_H at m = 3 for tol 1e-6),
    so a wrong constant or exponent in any of the three moves a threshold by
    far more than the 1e-5 margin used here."""
    assert oracle.quad_order(R * (1 + 1e-5), tol) == m, (tol, m, est)
    assert oracle.quad_order(R * (1 - 1e-5), tol) == m + 1, (tol, m, est)


def test_quad_order_cap_at_six():
    """Below R_5 the estimates would ask for m = 7 and more; the paper caps m at 6."""
    R5 = [r for (t, m, _, r) in order_thresholds_golden() if t == 1e-3 and m == 5][0]
    for rt in (R5 * (1 - 1e-5), 1.5, 1.31):
        assert oracle.quad_order(rt) == 6


# ------------------------------------------------------------------ kernels
def test_kernel_derivatives_match_finite_differences():
    rng = np.random.default_rng(7)
    k = 23.0
    for _ in range(5):
        x = rng.normal(size=3) * 0.05
        y = x + rng.normal(size=3) * 0.03
        nx = rng.normal(size=3); nx /= np.linalg.norm(nx)
        ny = rng.normal(size=3); ny /= np.linalg.norm(ny)
        G, H, Hp, E = oracle.kernels(x, nx, y, ny, k)
        h = 1e-4 * np.linalg.norm(y - x)

        def g(xx, yy):
            return oracle.kernels(xx, nx, yy, ny, k)[0]
        Hfd = (g(x, y + h * ny) - g(x, y - h * ny)) / (2 * h)
        Hpfd = (g(x + h * nx, y) - g(x - h * nx, y)) / (2 * h)
        Efd = (g(x + h * nx, y + h * ny) - g(x + h * nx, y - h * ny)
               - g(x - h * nx, y + h * ny) + g(x - h * nx, y - h * ny)) / (4 * h * h)
        assert abs(H - Hfd) < 1e-6 * abs(H) + 1e-9
        assert abs(Hp - Hpfd) < 1e-6 * abs(Hp) + 1e-9
        assert abs(E - Efd) < 1e-4 * abs(E) + 1e-6
        r = np.linalg.norm(y - x)
        assert abs(G - np.exp(1j * k * r) / (4 * np.pi * r)) < 1e-14 * abs(G)


# ------------------------------------------------------------------ singular rules
def _triangle():
    a = np.array([0.0, 0.0, 0.0]); b = np.array([0.011, 0.001, 0.0]); c = np.array([0.003, 0.009, 0.0])
    return a, b, c


def _hexagon(a, b, c):
    return np.array([a, (a + b) / 2, b, (b + c) / 2, c, (c + a) / 2])


def test_duffy_static_matches_polygon_closed_form():
    a, b, c = _triangle()
    x = (a + b + c) / 3
    exact = polygon_static_G(x, [a, b, c])
    assert abs(oracle.duffy_G(x, _hexagon(a, b, c), 0.0, n=24) - exact) < 1e-12 * exact
    # the paper's 4 x 4 rule
    assert abs(oracle.duffy_G(x, _hexagon(a, b, c), 0.0, n=4) - exact) < 2e-4 * exact


def test_edge_rule_static_matches_polygon_closed_form():
    a, b, c = _triangle()
    x = (a + b + c) / 3
    n = np.array([0.0, 0.0, 1.0])
    exact = polygon_static_E(x, [a, b, c])
    assert exact < 0
    assert abs(oracle.edge_fp(x, n, [a, b, c], 0.0, parts=64, ng=8) - exact) < 1e-11 * abs(exact)
    assert abs(oracle.edge_fp(x, n, [a, b, c], 0.0) - exact) < 2e-3 * abs(exact)


@pytest.mark.parametrize("k", [5.0, 73.0, 300.0])
def test_disk_limits_of_singular_rules(k):
    """On a fine regular polygon around x the Duffy G and the finite-part E
    (edge integral + k^2 G) tend to the disk closed forms."""
    R, nv = 0.004, 720
    th = 2 * np.pi * np.arange(nv) / nv
    poly = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(nv)], axis=1)
    x = np.zeros(3)
    n = np.array([0.0, 0.0, 1.0])
    Gp = oracle.duffy_G(x, poly, k, n=8)
    Ep = oracle.edge_fp(x, n, poly, k, parts=1, ng=4) + k * k * Gp
    rel = 3.0 * (2 * np.pi / nv) ** 2      # polygon vs disk geometry
    assert abs(Gp - disk_G(k, R)) < rel * abs(disk_G(k, R))
    assert abs(Ep - disk_E(k, R)) < rel * abs(disk_E(k, R))


def test_self_term_against_independent_quadrature():
    """G_ii at k != 0: static closed form plus scipy's adaptive integral of the
    smooth remainder (e^{ikr} - 1)/(4 pi r); H_ii = H'_ii = 0."""
    a, b, c = _triangle()
    x = (a + b + c) / 3
    k = 150.0
    nx = np.array([0.0, 0.0, 1.0])
    out = oracle.element_integrals(x, nx, a, b, c, k, self_term=True)

    def rem(v, u, part):
        y = a + u * (b - a) + v * (c - a)
        r = np.linalg.norm(y - x)
        f = (np.exp(1j * k * r) - 1.0) / (4 * np.pi * r)
        return f.real if part == 0 else f.imag
    area2 = np.linalg.norm(np.cross(b - a, c - a))
    re = integrate.dblquad(rem, 0, 1, 0, lambda u: 1 - u, args=(0,), epsabs=1e-14)[0]
    im = integrate.dblquad(rem, 0, 1, 0, lambda u: 1 - u, args=(1,), epsabs=1e-14)[0]
    ref = polygon_static_G(x, [a, b, c]) + area2 * (re + 1j * im)
    assert abs(out[0] - ref) < 3e-4 * abs(ref)
    assert out[1] == 0 and out[2] == 0


def _brute(x, nx, a, b, c, k, which):
    ny = np.cross(b - a, c - a); area2 = np.linalg.norm(ny); ny = ny / area2

    def f(v, u, part):
        y = a + u * (b - a) + v * (c - a)
        val = oracle.kernels(x, nx, y, ny, k)[which]
        return val.real if part == 0 else val.imag
    re = integrate.dblquad(f, 0, 1, 0, lambda u: 1 - u, args=(0,), epsabs=1e-15, epsrel=1e-11)[0]
    im = integrate.dblquad(f, 0, 1, 0, lambda u: 1 - u, args=(1,), epsabs=1e-15, epsrel=1e-11)[0]
    return area2 * (re + 1j * im)


@pytest.mark.parametrize("dist", [0.004, 0.008, 0.02, 0.06])
def test_regular_and_quasi_singular_rules_meet_tolerance(dist):
    """Element integrals with the paper's subdivision + a-priori order reach
    the paper's 1e-3 target against scipy's adaptive quadrature."""
    a, b, c = _triangle()
    x = (a + b + c) / 3 + np.array([0.002, -0.001, dist])
    nx = np.array([0.3, 0.1, 0.9]); nx /= np.linalg.norm(nx)
    k = 40.0
    out = oracle.element_integrals(x, nx, a, b, c, k)
    for which in range(4):
        ref = _brute(x, nx, a, b, c, k, which)
        assert abs(out[which] - ref) < 1e-3 * abs(ref), which


def test_in_plane_neighbour_quasi_singular():
    """Collocation point in the plane, just outside an edge: needs several
    subdivision levels."""
    a, b, c = _triangle()
    x = np.array([0.005, -0.0015, 0.0])
    nx = np.array([0.0, 0.0, 1.0])
    k = 40.0
    out = oracle.element_integrals(x, nx, a, b, c, k)
    for which in (0, 3):
        ref = _brute(x, nx, a, b, c, k, which)
        assert abs(out[which] - ref) < 2e-3 * abs(ref), which
    assert abs(out[1]) < 1e-12 * abs(out[0]) * 1e3     # coplanar: H = 0


def test_subdivision_limit_reports_element():
    """Overlapping elements (a collocation point inside another element) hit
    the subdivision limit; the error names the element (Sec. 4.1)."""
    from paper_2312_00005_gb300 import inputs
    nodes, tris = inputs.icosphere(1, 0.1)
    tris = np.vstack([tris, tris[5:6]])           # element 80 duplicates element 5
    n = tris.shape[0]
    cp = np.ones(n, complex); cq = np.zeros(n, complex)
    with pytest.raises(oracle.OracleError) as e:
        oracle.assemble(nodes, tris, 10.0, cp, cq)
    assert e.value.element in (5, 80)


# ------------------------------------------------------------------ FMM pieces
@pytest.mark.parametrize("x", [0.3, 1.7, 9.0, 40.0])
def test_spherical_hankel(x):
    h = oracle.sph_hankel(30, x)
    for n in range(4):
        assert abs(h[n] - sph_hankel_closed(n, x)) < 1e-13 * abs(h[n])
    for n in range(31):
        ref = spherical_jn(n, x) + 1j * spherical_yn(n, x)
        assert abs(h[n] - ref) < 1e-9 * abs(ref)


def test_sphere_grid_integrates_plane_waves():
    L = 12
    s, w = oracle.sphere_grid(L)
    assert abs(w.sum() - 4 * np.pi) < 1e-12
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0)
    k = 1.0
    for d in ([0.0, 0.0, 3.0], [1.0, 2.0, -2.0], [4.0, -1.0, 1.0]):
        d = np.array(d)
        val = np.sum(w * np.exp(1j * k * s @ d))
        ref = 4 * np.pi * spherical_jn(0, k * np.linalg.norm(d))
        assert abs(val - ref) < 1e-9


def test_single_pair_expansion_reproduces_green_function():
    """Eq. FMMBase with prefactor ik/(16 pi^2) converges to G(x, y) as L
    grows past k|z1 - z2|, and becomes unstable once h_L(k|z1 - z2|) is huge
    (the small-argument Hankel growth of Sec. 4.2)."""
    k = 60.0
    z1 = np.array([0.0, 0.0, 0.0]); z2 = np.array([0.07, 0.02, -0.05])
    x = z1 + np.array([0.004, -0.003, 0.002]); y = z2 + np.array([-0.002, 0.005, 0.001])
    r = np.linalg.norm(x - y)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    errs = {L: abs(oracle.fmm_pair(x, y, z1, z2, k, L) - G) / abs(G) for L in (4, 8, 12, 30)}
    assert errs[4] > errs[8] > errs[12]
    assert errs[12] < 1e-10
    assert errs[30] > 1.0
