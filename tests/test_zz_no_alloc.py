"""The no-allocation entry point (bem_matvec_direct_noalloc) against the
regular direct product (bem_matvec on a mesh in direct mode).

The entry point exists for callers that may not allocate device memory while
running (its element data live in a fixed array inside the library), so it
takes the mesh as caller-owned device arrays.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2312_00005_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, RHO = 343.0, 1.21


@pytest.fixture(scope="module")
def bem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_00005_gb300 import bemfmm
    bemfmm.lib()
    return bemfmm


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_direct_product_on_two_calls(bem):
    """Two calls in a row (different meshes and vectors, so the second call
    reuses the scratch the first one wrote) agree with bem_matvec within the
    direct-product tolerance of the parity tests (2e-5)."""
    cases = [(inputs.icosphere(3, 0.1), 1500.0, 31), (inputs.bumpy_ellipsoid(9), 2500.0, 32)]
    for (nodes, tris), freq, seed in cases:
        n = tris.shape[0]
        x = inputs.random_complex(n, seed)
        xt = torch.tensor(x, dtype=torch.complex64, device="cuda")
        mesh = bem.Mesh(nodes, tris, mode=bem.MODE_DIRECT)
        y_ref = mesh.matvec(freq, xt, c=C, rho=RHO).cpu().numpy()
        mesh.close()
        nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
        td = torch.tensor(tris, dtype=torch.int32, device="cuda")
        y = torch.empty_like(xt)
        bem.matvec_direct_noalloc(nd, td, freq, xt, y, c=C, rho=RHO)
        err = _rel(y.cpu().numpy(), y_ref)
        assert err < 2e-5, (n, err)


def test_noalloc_rejects_meshes_above_its_limit(bem):
    nodes, tris = inputs.icosphere(1, 0.1)
    nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
    td = torch.zeros((40000, 3), dtype=torch.int32, device="cuda")
    x = torch.zeros(40000, dtype=torch.complex64, device="cuda")
    with pytest.raises(bem.BemError) as e:
        bem.matvec_direct_noalloc(nd, td, 1000.0, x, torch.empty_like(x))
    assert e.value.code == -1 and "32768" in str(e.value)
