"""The no-allocation entry point (bem_matvec_direct_noalloc) against the
FP64 oracle's dense operator and against the regular direct product
(bem_matvec on a mesh in direct mode).

The entry point exists for callers that may not allocate device memory while
running (its element data live in a fixed array inside the library), so it
takes the mesh as caller-owned device arrays.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2312_00005_gb300 import inputs

torch = pytest.importorskip("torch")

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


def _elem(a, b):
    s = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
    return float(np.max(np.abs(a - b) / s))


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_direct_product_on_two_calls(bem):
    """Two calls in a row (different meshes and vectors, so the second call
    reuses the scratch the first one wrote) agree with the oracle's dense
    sound-hard operator (Eq. SystemI with every pair by the quadrature of
    Sec. 3.1) within the direct-product tolerance of the parity tests (2e-5
    relative l2, 2e-4 per element), and with bem_matvec in direct mode."""
    cases = [(inputs.icosphere(3, 0.1), 1500.0, 31), (inputs.bumpy_ellipsoid(9), 2500.0, 32)]
    for (nodes, tris), freq, seed in cases:
        n = tris.shape[0]
        k = 2 * np.pi * freq / C
        x = inputs.random_complex(n, seed)
        xt = torch.tensor(x, dtype=torch.complex64, device="cuda")
        nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
        td = torch.tensor(tris, dtype=torch.int32, device="cuda")
        y = torch.empty_like(xt)
        bem.matvec_direct_noalloc(nd, td, freq, xt, y, c=C, rho=RHO)
        yn = y.cpu().numpy()
        yo = oracle.assemble(nodes, tris, k, np.ones(n, complex), np.zeros(n, complex)) @ x
        assert _rel(yn, yo) < 2e-5 and _elem(yn, yo) < 2e-4, (n, _rel(yn, yo), _elem(yn, yo))
        mesh = bem.Mesh(nodes, tris, mode=bem.MODE_DIRECT)
        y_ref = mesh.matvec(freq, xt, c=C, rho=RHO).cpu().numpy()
        mesh.close()
        assert _rel(yn, y_ref) < 2e-5, (n, _rel(yn, y_ref))


@pytest.mark.gpu
def test_noalloc_rejects_meshes_above_its_limit(bem):
    nodes, tris = inputs.icosphere(1, 0.1)
    nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
    td = torch.zeros((40000, 3), dtype=torch.int32, device="cuda")
    x = torch.zeros(40000, dtype=torch.complex64, device="cuda")
    with pytest.raises(bem.BemError) as e:
        bem.matvec_direct_noalloc(nd, td, 1000.0, x, torch.empty_like(x))
    assert e.value.code == -1 and "32768" in str(e.value)


@pytest.mark.gpu
def test_noalloc_binding_rejects_wrong_shapes_before_any_launch(bem):
    """The C entry point cannot see shapes; the binding rejects a flat tris
    tensor, a tris tensor of width 2, nodes without three coordinates and
    vectors of the wrong length (each would make the kernels read past the
    caller's buffers)."""
    nodes, tris = inputs.icosphere(1, 0.1)
    n = tris.shape[0]
    nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
    td = torch.tensor(tris, dtype=torch.int32, device="cuda")
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    bad = [(nd, td.reshape(-1), x, y), (nd, td[:, :2].contiguous(), x, y), (nd.reshape(-1), td, x, y),
           (nd, td, x[:-1], y[:-1]), (nd, td, torch.zeros(n + 1, dtype=torch.complex64, device="cuda"), y)]
    before = bem.launch_count()
    for a in bad:
        with pytest.raises(ValueError):
            bem.matvec_direct_noalloc(a[0], a[1], 1000.0, a[2], a[3])
    assert bem.launch_count() == before


@pytest.mark.gpu
def test_noalloc_medium_defaults_as_the_mesh_entry_points(bem):
    """c <= 0 means 343 m/s, as for bem_mesh_create's entry points."""
    nodes, tris = inputs.icosphere(2, 0.1)
    n = tris.shape[0]
    nd = torch.tensor(nodes, dtype=torch.float64, device="cuda")
    td = torch.tensor(tris, dtype=torch.int32, device="cuda")
    x = torch.tensor(inputs.random_complex(n, 3), dtype=torch.complex64, device="cuda")
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    bem.matvec_direct_noalloc(nd, td, 1200.0, x, y0, c=343.0)
    bem.matvec_direct_noalloc(nd, td, 1200.0, x, y1, c=0.0)
    assert torch.equal(y0, y1)


def test_noalloc_binding_rejects_host_tensors():
    """Host-side: tensors that are not on a CUDA device are refused before
    the library is called."""
    from paper_2312_00005_gb300 import bemfmm
    nodes, tris = inputs.icosphere(1, 0.1)
    x = torch.zeros(tris.shape[0], dtype=torch.complex64)
    with pytest.raises(TypeError):
        bemfmm.matvec_direct_noalloc(torch.tensor(nodes), torch.tensor(tris, dtype=torch.int32), 1000.0, x, x)
