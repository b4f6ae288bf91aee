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
