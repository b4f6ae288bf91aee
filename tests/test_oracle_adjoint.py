"""Pins of the oracle's adjoint gradient of a field loss with respect to the
region admittances (L = sum_m |p(x_m)|^2, p the total field of Eq. BIE_I at
points x_m, the surface solution from Eq. SystemI with the admittance
condition q = -tau i k rho c Y p on each region).

The gradient is checked against central finite differences of the forward
oracle (solve + field) for the exterior and the interior (tau = -1) problem
with mixed boundary conditions, and against the derivative of the
admittance-sphere series (closed form, independent of the oracle)."""
import numpy as np
import pytest

import oracle
from closed_forms import sphere_plane_wave, sphere_plane_wave_dbeta
from paper_2312_00005_gb300 import inputs

C, RHO, A = 343.0, 1.21, 0.1
PLANE_Z = [("plane", (0.0, 0.0, 1.0), 1.0)]


def _octants(cen, centre=(0.0, 0.0, 0.0)):
    d = cen - np.asarray(centre)
    return ((d[:, 0] > 0) + 2 * (d[:, 1] > 0) + 4 * (d[:, 2] > 0)).astype(np.int64)


def _passive_Y(nreg, seed, rho=RHO, c=C):
    """beta = rho c Y = r e^{i phi}, r ~ U(0, 0.5), phi ~ U(-pi/2, pi/2)."""
    rng = np.random.default_rng(seed)
    beta = rng.uniform(0.0, 0.5, nreg) * np.exp(1j * rng.uniform(-np.pi / 2, np.pi / 2, nreg))
    return beta / (rho * c)


def _loss(nodes, tris, f, pts, region, Y, sources, bc_type, bc_value=None, c=C, rho=RHO, params=None):
    """Forward loss from the pinned forward oracle (solve, then field)."""
    n = tris.shape[0]
    beta = np.zeros(n, np.complex128)
    adm = bc_type == oracle.ADMI
    beta[adm] = rho * c * np.asarray(Y)[region[adm]]
    p, q, info = oracle.solve(nodes, tris, f, c=c, rho=rho, sources=sources, bc_type=bc_type,
                              bc_value=bc_value, beta=beta, tol=1e-13, params=params)
    assert info["converged"]
    fld = oracle.field(nodes, tris, f, p, q, pts, c=c, sources=sources, params=params)
    return float(np.sum(np.abs(fld) ** 2))


def _central_differences(loss, Y, rel=1e-6):
    g = np.zeros(Y.shape[0], np.complex128)
    for r in range(Y.shape[0]):
        h = rel * abs(Y[r])
        e = np.zeros(Y.shape[0])
        e[r] = 1.0
        dre = (loss(Y + h * e) - loss(Y - h * e)) / (2 * h)
        dim = (loss(Y + 1j * h * e) - loss(Y - 1j * h * e)) / (2 * h)
        g[r] = dre + 1j * dim
    return g


def test_series_derivative_matches_difference_quotient():
    """The closed-form dp/dbeta against a difference quotient of the series."""
    k = 2 * np.pi * 1000.0 / C
    pts = inputs.fibonacci_sphere(20, 1.0)
    for beta in (0.3 + 0.2j, 0.05 - 0.4j):
        h = 1e-6
        fd = (sphere_plane_wave(pts, k, A, beta + h) - sphere_plane_wave(pts, k, A, beta - h)) / (2 * h)
        cf = sphere_plane_wave_dbeta(pts, k, A, beta)
        assert np.max(np.abs(fd - cf)) < 1e-7 * np.max(np.abs(cf))


def test_adjoint_matches_finite_differences_exterior():
    """Eight octant regions on a 320-element sphere with passive admittances,
    a plane wave and a point source; one unused region has zero gradient."""
    nodes, tris = inputs.icosphere(2, A)
    cen, _, _ = oracle.geometry(nodes, tris)
    region = _octants(cen)
    Y = np.concatenate([_passive_Y(8, 2312), [0.001 + 0.0005j]])
    f = 1000.0
    src = PLANE_Z + [("point", (0.0, 0.13, 0.02), 0.5 - 0.2j)]
    pts = inputs.fibonacci_sphere(20, 1.0)
    bct = np.full(tris.shape[0], oracle.ADMI, np.int32)
    L, g, info = oracle.admittance_gradient(nodes, tris, f, pts, region, Y, sources=src)
    assert info["forward"]["converged"] and info["adjoint"]["converged"]
    assert g[8] == 0
    loss = lambda y: _loss(nodes, tris, f, pts, region, y, src, bct)
    assert abs(L - loss(Y)) < 1e-10 * L
    fd = _central_differences(loss, Y[:8])
    assert np.max(np.abs(fd - g[:8])) < 1e-5 * np.max(np.abs(g[:8]))


def test_system_is_linear_in_column_coefficients():
    """Step 1 of the adjoint: A(cp, cq) = Ap diag(cp) + Aq diag(cq)."""
    nodes, tris = inputs.icosphere(1, A)
    n = tris.shape[0]
    k = 2 * np.pi * 1500.0 / C
    rng = np.random.default_rng(5)
    cp = rng.normal(size=n) + 1j * rng.normal(size=n)
    cq = rng.normal(size=n) + 1j * rng.normal(size=n)
    ones, zeros = np.ones(n, np.complex128), np.zeros(n, np.complex128)
    for params in (None, {"tau": -1.0}):
        Ap = oracle.assemble(nodes, tris, k, ones, zeros, params)
        Aq = oracle.assemble(nodes, tris, k, zeros, ones, params)
        Afull = oracle.assemble(nodes, tris, k, cp, cq, params)
        assert np.max(np.abs(Ap * cp[None, :] + Aq * cq[None, :] - Afull)) < 1e-13 * np.max(np.abs(Afull))


def test_adjoint_matches_finite_differences_interior():
    """Interior problem (tau = -1) in a short closed duct: driven end
    (velocity), admittance regions on the far end and the two halves of the
    side walls, field points on the axis."""
    c, rho, f = 340.0, 1.3, 240.0
    nodes, tris = inputs.duct(0.6, 0.2, 0.1)
    cen, _, _ = oracle.geometry(nodes, tris)
    drive = cen[:, 0] < 1e-9
    far = cen[:, 0] > 0.6 - 1e-9
    assert drive.sum() == far.sum() == 8
    region = np.where(far, 0, np.where(cen[:, 2] < 0, 1, 2)).astype(np.int64)
    region[drive] = -1
    bct = np.where(drive, oracle.VELO, oracle.ADMI).astype(np.int32)
    bcv = np.where(drive, 1.0, 0.0).astype(np.complex128)
    Y = np.array([1.0 / (rho * c), 0.2 / (rho * c) * np.exp(0.3j), 0.1 / (rho * c) * np.exp(-0.5j)])
    xs = np.linspace(0.1, 0.5, 5)
    pts = np.stack([xs, 0 * xs + 0.01, 0 * xs - 0.02], 1)
    params = {"tau": -1.0}
    L, g, info = oracle.admittance_gradient(nodes, tris, f, pts, region, Y, bc_type=bct, bc_value=bcv,
                                            c=c, rho=rho, params=params)
    assert info["forward"]["converged"] and info["adjoint"]["converged"]
    loss = lambda y: _loss(nodes, tris, f, pts, region, y, (), bct, bcv, c=c, rho=rho, params=params)
    assert abs(L - loss(Y)) < 1e-10 * L
    fd = _central_differences(loss, Y)
    assert np.max(np.abs(fd - g)) < 1e-5 * np.max(np.abs(g))


def test_adjoint_matches_sphere_series():
    """Uniform admittance beta = 0.3 + 0.2i on the whole sphere: the gradient
    of the loss at 20 points on a 1 m sphere against the series derivative
    (dL/dY = rho c dL/dbeta), within the discretisation error, which falls
    with refinement.  Split into eight regions with equal Y, the region
    gradients add up to the single-region gradient (chain rule)."""
    f = 1000.0
    k = 2 * np.pi * f / C
    beta = 0.3 + 0.2j
    pts = inputs.fibonacci_sphere(20, 1.0)
    fs = sphere_plane_wave(pts, k, A, beta)
    dfs = RHO * C * sphere_plane_wave_dbeta(pts, k, A, beta)
    g_series = 2.0 * np.conj(np.vdot(fs, dfs))
    L_series = float(np.sum(np.abs(fs) ** 2))
    errs = []
    for lev in (2, 3):
        nodes, tris = inputs.icosphere(lev, A)
        n = tris.shape[0]
        L, g, _ = oracle.admittance_gradient(nodes, tris, f, pts, np.zeros(n, np.int64), [beta / (RHO * C)],
                                             sources=PLANE_Z)
        assert abs(L - L_series) < 1e-3 * L_series
        errs.append(abs(g[0] - g_series) / abs(g_series))
        if lev == 2:
            cen, _, _ = oracle.geometry(nodes, tris)
            _, g8, _ = oracle.admittance_gradient(nodes, tris, f, pts, _octants(cen),
                                                  np.full(8, beta / (RHO * C)), sources=PLANE_Z)
            assert abs(g8.sum() - g[0]) < 1e-9 * abs(g[0])
    assert errs[1] < 0.025, errs             # 3.1% at 320, 1.4% at 1280 elements
    assert errs[1] < errs[0] / 1.6, errs
    # the opposite admittance sign is far off
    fw = sphere_plane_wave(pts, k, A, -beta)
    g_wrong = 2.0 * np.conj(np.vdot(fw, RHO * C * sphere_plane_wave_dbeta(pts, k, A, -beta)))
    assert abs(g_wrong - g_series) > 5 * errs[1] * abs(g_series)


@pytest.mark.parametrize("bad", [[-1], [3]])
def test_adjoint_rejects_unmapped_admittance_elements(bad):
    nodes, tris = inputs.icosphere(1, A)
    n = tris.shape[0]
    region = np.zeros(n, np.int64)
    region[0] = bad[0]
    bct = np.full(n, oracle.ADMI, np.int32)
    with pytest.raises(ValueError):
        oracle.admittance_gradient(nodes, tris, 1000.0, inputs.fibonacci_sphere(4, 1.0), region,
                                   [0.001], sources=PLANE_Z, bc_type=bct)
