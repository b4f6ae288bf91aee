"""The synthetic meshes are closed, consistently wound surfaces with the
stated sizes: total area, and the divergence theorem (the flux of x through
the surface is three times the enclosed volume, positive only when every
triangle is wound out of the volume)."""
import numpy as np
import pytest

from paper_2312_00005_gb300 import inputs


def _area_and_flux(nodes, tris):
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    flux = np.einsum("ij,ij->i", 0.5 * cr, (a + b + c) / 3.0).sum()
    return area, flux


@pytest.mark.parametrize("h", [0.1, 0.05])
def test_duct_is_closed_and_wound_outward(h):
    L, w = 3.4, 0.2
    nodes, tris = inputs.duct(L, w, h)
    nx, ny = round(L / h), round(w / h)
    assert tris.shape[0] == 2 * (4 * nx * ny + 2 * ny * ny)
    area, flux = _area_and_flux(nodes, tris)
    assert np.isclose(area.sum(), 4 * L * w + 2 * w * w, rtol=1e-12)
    assert np.isclose(flux, 3 * L * w * w, rtol=1e-12)
    # halves of the face grids' rectangles: side faces (L / nx) x (w / ny), ends (w / ny)^2
    side = np.isclose(area, 0.5 * (L / nx) * (w / ny), rtol=1e-9)
    end = np.isclose(area, 0.5 * (w / ny) ** 2, rtol=1e-9)
    assert np.all(side | end)


def test_icosphere_is_closed_and_wound_outward():
    nodes, tris = inputs.icosphere(3, 0.1)
    assert tris.shape[0] == 20 * 4 ** 3
    area, flux = _area_and_flux(nodes, tris)
    # inscribed polyhedron: slightly below the sphere's area and volume
    assert 0.99 * 4 * np.pi * 0.01 < area.sum() < 4 * np.pi * 0.01
    assert 0.98 * 4 * np.pi * 0.001 < flux < 4 * np.pi * 0.001


def test_head_bands_cover_the_sweep_with_fine_enough_meshes():
    """64 frequencies 200 Hz .. 16 kHz in bands of increasing mesh size; each
    band's mean edge is at most min(lambda / 10.7, 11 mm) at its highest
    frequency; N from about 2.4k to about 70k; the point source lies 1 mm
    outside the surface."""
    bands = inputs.head_bands()
    freqs = np.concatenate([f for _, f in bands])
    assert freqs.shape[0] == 64
    assert abs(freqs[0] - 200.0) < 1e-9 and abs(freqs[-1] - 16000.0) < 1e-6
    assert np.all(np.diff(freqs) > 0)
    nus = [nu for nu, _ in bands]
    assert nus == sorted(nus) and len(set(nus)) == len(nus)
    assert 20 * nus[0] ** 2 < 3000 and 60000 < 20 * nus[-1] ** 2 < 80000
    for nu, f in (bands[0], bands[len(bands) // 2]):
        nodes, tris = inputs.bumpy_ellipsoid(nu)
        e = np.concatenate([np.linalg.norm(nodes[tris[:, a]] - nodes[tris[:, b]], axis=1)
                            for a, b in ((0, 1), (1, 2), (2, 0))])
        assert e.mean() <= min(343.0 / max(f) / 10.7, 0.011) * (1 + 1e-9)
    nodes, tris = inputs.bumpy_ellipsoid(30)
    xs = inputs.head_point_source()
    d = np.linalg.norm(nodes - xs, axis=1).min()
    assert 0.0009 < d < 0.0011
    assert xs[1] > nodes[:, 1].max()
