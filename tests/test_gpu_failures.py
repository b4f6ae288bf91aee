"""Failure paths of the library on the GPU, reached without a GPU fault
(bem_test_hooks): a device allocation that fails must come back as an error
code, leave the mesh usable and leak no device memory.  (No kernel of the
library waits on another block or launch; the one device wait, the
tensor-core aggregation's bounded wait for its own MMAs, is not forced to
give up, since that would free tensor memory under MMAs in flight.)"""
import numpy as np
import pytest

import oracle
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
    bemfmm.test_hooks()
    yield bemfmm
    bemfmm.test_hooks()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_allocation_failure_reports_oom_without_leaking(bem):
    """Every device allocation of mesh creation and of an FMM solve is made
    to fail in turn: each failure is BEM_E_OOM (never a crash or another
    code), and once the meshes are destroyed the library holds exactly the
    device memory it held before."""
    nodes, tris = inputs.icosphere(4, 0.1)       # FMM path: plan, tables, near field, GMRES
    src = [bem.plane_wave((0, 0, 1))]
    live0 = bem.test_hooks()
    failures, ok = 0, False
    for after in range(0, 400, 3):
        bem.test_hooks(alloc_fail_after=after)
        mesh = None
        try:
            mesh = bem.Mesh(nodes, tris, trunc_factor=5.0)
            mesh.solve(2000.0, src, tol=1e-6, c=C, rho=RHO)
            ok = True
        except bem.BemError as e:
            assert e.code == -4, (after, str(e))
            assert "refused by the test hook" in str(e)
            failures += 1
        finally:
            bem.test_hooks()
            if mesh is not None:
                mesh.close()
        assert bem.test_hooks() == live0, after
        if ok:
            break
    assert ok and failures >= 5, (ok, failures)
    # a mesh whose solve failed on an allocation still solves afterwards
    mesh = bem.Mesh(nodes, tris, trunc_factor=5.0)
    bem.test_hooks(alloc_fail_after=2)
    try:
        with pytest.raises(bem.BemError):
            mesh.solve(2000.0, src, tol=1e-6, c=C, rho=RHO)
    finally:
        bem.test_hooks()
    p, q, info = mesh.solve(2000.0, src, tol=1e-6, c=C, rho=RHO)
    assert info["converged"], info
    mesh.close()
    assert bem.test_hooks() == live0
