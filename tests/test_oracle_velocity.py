"""Pins of the oracle's particle velocity at field points, v = grad p /
(i w rho) (Eq. utopandv), with grad p from Eq. BIE_I (lambda = 1)
differentiated under the integral: central differences of the oracle's own
field (itself pinned against the sphere series), and the plane wave's
velocity, which is the wave's pressure over the impedance rho c along its
direction."""
import numpy as np

import oracle
from paper_2312_00005_gb300 import inputs

C, RHO = 343.0, 1.21


def test_plane_wave_velocity_is_pressure_over_impedance():
    # with p = q = 0 on the surface only the incident wave remains
    nodes, tris = inputs.icosphere(1, 0.1)
    n = tris.shape[0]
    f = 700.0
    k = 2 * np.pi * f / C
    pts = np.array([[0.5, 0.1, -0.2], [0.0, 0.8, 0.3], [-0.4, -0.4, 0.6]])
    z = np.zeros(n, complex)
    d = np.array([0.3, -0.2, 0.93])
    d /= np.linalg.norm(d)
    amp = 0.7 - 0.2j
    v = oracle.field_velocity(nodes, tris, f, z, z, pts, c=C, rho=RHO, sources=[("plane", d, amp)])
    p = amp * np.exp(1j * k * pts @ d)
    np.testing.assert_allclose(v, p[:, None] * d[None, :] / (RHO * C), rtol=1e-12, atol=1e-15)


def test_velocity_matches_central_differences_of_the_field():
    """Seeded surface data p, q (both terms of Eq. BIE_I matter), a plane
    wave and a point source, points from 0.16 m to 0.9 m off a 0.1 m sphere
    (regular rules of order 1 to 3): the analytic gradient of the oracle's
    field equals its central difference with step 1e-6 m (truncation and
    rounding both far below the tolerance)."""
    nodes, tris = inputs.icosphere(2, 0.1)
    n = tris.shape[0]
    f = 800.0
    rng = np.random.default_rng(5)
    p = rng.normal(size=n) + 1j * rng.normal(size=n)
    q = (rng.normal(size=n) + 1j * rng.normal(size=n)) * 10.0
    src = [("plane", (0.0, 0.6, 0.8), 1.0 + 0.5j), ("point", (0.02, -0.01, 0.03), 0.4 - 0.3j)]
    pts = np.array([[0.6, 0.3, 0.7], [0.0, -0.25, 0.12], [0.13, 0.1, -0.2]])
    v = oracle.field_velocity(nodes, tris, f, p, q, pts, c=C, rho=RHO, sources=src)
    grad = v * (1j * 2 * np.pi * f * RHO)
    h = 1e-6
    fd = np.zeros((pts.shape[0], 3), complex)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fp = oracle.field(nodes, tris, f, p, q, pts + e, c=C, sources=src)
        fm = oracle.field(nodes, tris, f, p, q, pts - e, c=C, sources=src)
        fd[:, ax] = (fp - fm) / (2 * h)
    err = np.linalg.norm(grad - fd) / np.linalg.norm(fd)
    assert err < 1e-6, err
    # each point and axis on its own, so that no component hides behind a larger one
    rel = np.abs(grad - fd) / np.abs(fd).max(axis=1, keepdims=True)
    assert rel.max() < 1e-6, rel
