"""The mixed-precision form (bem_params.far_precision = 1): the aggregation
of Sec. 3.3.3 (T(l)) on the tensor cores in split BF16 (tcgen05, three BF16
products accumulated in FP32), and the FP64 iterative refinement that gives
its solves the FP32 form's accuracy.  Against the FP32 form (far_precision
0) on the same inputs and against the FP64 oracle."""
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
    return bemfmm


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _elem(a, b):
    s = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
    return float(np.max(np.abs(a - b) / s))


def _check(a, b, l2, el, what):
    e2, ee = _rel(a, b), _elem(a, b)
    print("%s: rel l2 %.3g (bound %.0e), per element %.3g (bound %.0e)" % (what, e2, l2, ee, el))
    assert e2 < l2 and ee < el, (what, e2, ee)


def _mixed_bc(n, seed):
    rng = np.random.default_rng(seed)
    bct = rng.integers(0, 3, n).astype(np.int32)
    region = rng.integers(0, 4, n).astype(np.int32)
    adm = (rng.uniform(0, 0.5, 4) * np.exp(1j * rng.uniform(-1.5, 1.5, 4))) / (RHO * C)
    return bct, region, adm


@pytest.mark.parametrize("nrhs", [1, 4])
def test_tensor_core_products_match_fp32_form_and_oracle(bem, nrhs):
    """Products with the split-BF16 tensor-core aggregation (5120 elements,
    2 kHz, three far levels, mixed boundary conditions, 1 and 4 right-hand
    sides) against the FP32 form and the oracle's dense operator.  The split
    keeps about 16 bits of each operand, so the products differ from the
    FP32 form by a few 1e-7 of the product (the far part is a fraction of
    it); the bounds leave a factor of ten."""
    nodes, tris = inputs.icosphere(4, 0.1)
    n = tris.shape[0]
    freq = 2000.0
    k = 2 * np.pi * freq / C
    bct, region, adm = _mixed_bc(n, 7)
    beta = RHO * C * adm[region]
    cp, cq, _, _ = oracle.column_coeffs(bct, k, C, RHO, beta)
    A = oracle.assemble(nodes, tris, k, cp, cq)
    X = np.stack([inputs.random_complex(n, 60 + r) for r in range(nrhs)])
    Yo = X @ A.T
    Xt = torch.tensor(X if nrhs > 1 else X[0], dtype=torch.complex64, device="cuda")
    Y = {}
    for fp in (0, 1):
        mesh = bem.Mesh(nodes, tris, bc_type=bct, region=region, trunc_factor=6.0, far_precision=fp)
        assert mesh.stats(freq, c=C)["levels"] >= 2
        Y[fp] = mesh.matvec(freq, Xt, admittance=adm, c=C, rho=RHO).cpu().numpy().reshape(nrhs, n)
        mesh.close()
    for r in range(nrhs):
        _check(Y[1][r], Y[0][r], 1e-5, 1e-4, "tensor-core vs FP32 aggregation, rhs %d of %d" % (r, nrhs))
        _check(Y[1][r], Yo[r], 1e-4, 1e-3, "tensor-core product vs oracle, rhs %d of %d" % (r, nrhs))


def test_mixed_precision_refined_solve_matches_oracle(bem):
    """bem_solve_multi with the tensor-core aggregation: three plane waves
    on a sphere with admittance data; the FP64 refinement (residuals with
    the FP32 products) reaches tol 1e-6 of the true residual, and the
    solutions match the FP32 form's and the oracle's."""
    nodes, tris = inputs.icosphere(4, 0.1)
    n = tris.shape[0]
    freq = 2000.0
    cen, _, _ = oracle.geometry(nodes, tris)
    bc = np.where(cen[:, 2] > 0.03, bem.ADMI, bem.VELO).astype(np.int32)
    region = np.zeros(n, np.int32)
    adm = np.array([0.3 * (1 - 0.2j)]) / (RHO * C)
    dirs = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, -0.6, 0.8)]
    src = [bem.plane_wave(d) for d in dirs]
    P = {}
    for fp in (0, 1):
        mesh = bem.Mesh(nodes, tris, bc_type=bc, region=region, trunc_factor=6.0, far_precision=fp)
        P[fp], _, infos = mesh.solve_multi(freq, src, admittance=adm, tol=1e-6, c=C, rho=RHO)
        mesh.close()
        assert all(i["converged"] for i in infos), infos
        print("far_precision", fp, "products", [i["iterations"] for i in infos], "relres",
              [i["relres"] for i in infos])
        if fp == 1:
            assert all(i["relres"] <= 1e-6 for i in infos), infos
    for r, d in enumerate(dirs):
        po, _, _ = oracle.solve(nodes, tris, freq, c=C, rho=RHO, sources=[("plane", d, 1.0)], bc_type=bc,
                                beta=RHO * C * adm[region])
        _check(P[1][r].cpu().numpy(), P[0][r].cpu().numpy(), 2e-5, 2e-4, "mixed vs FP32 form, rhs %d" % r)
        _check(P[1][r].cpu().numpy(), po, 2e-4, 2e-3, "mixed-precision solve vs oracle, rhs %d" % r)


@pytest.mark.parametrize("fp", [0, 1])
def test_far_field_reciprocity_of_multi_rhs_solves(bem, fp):
    """Reciprocity of the far-field amplitudes of plane-wave scattering,
    f(a -> -b) = f(b -> -a), for the four tetrahedral directions solved
    together (bem_solve_multi) on the bumpy head-like surface (10580
    elements, 5 kHz, block-Jacobi), in the FP32 form and in the
    mixed-precision form: the scattered fields at 50 m agree pairwise within
    the discretisation error (the identity holds for the continuum problem;
    the mesh resolves a thirteenth of the wavelength, about 1% error)."""
    nodes, tris = inputs.bumpy_ellipsoid(23)
    freq = 5000.0
    dirs = inputs.tetrahedral_directions()
    src = [bem.plane_wave(tuple(d)) for d in dirs]
    mesh = bem.Mesh(nodes, tris, trunc_factor=6.0, block_jacobi=1, restart=400, far_precision=fp)
    P, Q, infos = mesh.solve_multi(freq, src, tol=1e-6, max_iter=800, c=C, rho=RHO)
    assert all(i["converged"] for i in infos), infos
    amp = np.zeros((4, 4), complex)
    for a in range(4):
        amp[a] = mesh.evaluate(freq, P[a], Q[a], -50.0 * dirs, [], c=C, rho=RHO).cpu().numpy()
    mesh.close()
    rec = max(abs(amp[a, b] - amp[b, a]) / max(abs(amp[a, b]), abs(amp[b, a])) for a in range(4) for b in range(a + 1, 4))
    print("far_precision", fp, "products", [i["iterations"] for i in infos], "reciprocity", rec)
    assert rec < 0.05, rec
