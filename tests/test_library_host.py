"""CPU checks of the CUDA library: it builds for sm_103a, loads, exports
every entry point declared in include/*.h, and its host-side plan (Sec. 3.3.4
near / interaction lists) covers every element pair exactly once."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2312_00005_gb300 import bemfmm, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(bem_[a-z_0-9]+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2312_00005_gb300 import build
    build.build()
    return bemfmm.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"bem_mesh_create", "bem_matvec", "bem_solve", "bem_evaluate", "bem_last_error"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_params_default_are_the_papers(lib):
    p = bemfmm.default_params()
    assert p.quad_tol == 1e-3 and p.m_max == 6 and p.rt_subdiv == 1.3 and p.max_depth == 15
    assert p.trunc_factor == 1.8 and p.L_min == 8
    assert abs(p.admissibility - 2 / np.sqrt(3)) < 1e-15
    assert p.tau == 1.0          # exterior problem unless asked otherwise
    assert p.row_scaling == 0    # no preconditioner unless asked (Sec. 3.2: an option)
    assert p.far_table == 0      # phases of T and S regenerated in every product (faster on this GPU)
    assert p.graphs == 1         # each GMRES restart cycle one graph launch
    assert p.near_transpose == 1 # A^T stored for the transposed product


@pytest.mark.parametrize("rs", [-1, 2])
def test_row_scaling_other_than_zero_or_one_is_rejected(lib, rs):
    nodes, tris = inputs.icosphere(1, 0.1)
    with pytest.raises(bemfmm.BemError):
        bemfmm.Mesh(nodes, tris, row_scaling=rs)


@pytest.mark.parametrize("ft", [-1, 2])
def test_far_table_other_than_zero_or_one_is_rejected(lib, ft):
    nodes, tris = inputs.icosphere(1, 0.1)
    with pytest.raises(bemfmm.BemError, match="far_table"):
        bemfmm.Mesh(nodes, tris, far_table=ft)


@pytest.mark.parametrize("v", [-1, 2])
def test_near_transpose_other_than_zero_or_one_is_rejected(lib, v):
    nodes, tris = inputs.icosphere(1, 0.1)
    with pytest.raises(bemfmm.BemError, match="near_transpose"):
        bemfmm.Mesh(nodes, tris, near_transpose=v)


@pytest.mark.parametrize("g", [-1, 2])
def test_graphs_other_than_zero_or_one_is_rejected(lib, g):
    nodes, tris = inputs.icosphere(1, 0.1)
    with pytest.raises(bemfmm.BemError, match="graphs"):
        bemfmm.Mesh(nodes, tris, graphs=g)


@pytest.mark.parametrize("tau", [0.0, 0.5, -2.0, float("nan")])
def test_tau_other_than_plus_or_minus_one_is_rejected(lib, tau):
    """tau selects the exterior (+1) or interior (-1) problem of Eq. BIE_I;
    anything else is an argument error, raised before any device work."""
    nodes, tris = inputs.icosphere(1, 0.1)
    with pytest.raises(bemfmm.BemError):
        bemfmm.Mesh(nodes, tris, tau=tau)


@pytest.mark.parametrize("lev,freq", [(3, 1000.0), (4, 2000.0), (5, 4000.0)])
def test_plan_partitions_all_pairs(lib, lev, freq):
    nodes, tris = inputs.icosphere(lev, 0.1)
    n = tris.shape[0]
    st = bemfmm.plan_stats_host(nodes, tris, freq)
    assert st["near_nnz"] + st["far_pairs"] == n * n
    assert 0 <= st["asymmetric_pairs"] < 0.03 * n * n
    assert st["near_nnz"] >= n                  # the diagonal is near
    for L in st["L"]:
        assert L >= 8


def test_plan_with_parallel_list_building_partitions_all_pairs(lib):
    """69,620 elements at 16 kHz (leaf depth 6, 12,416 leaves): the list
    builder scans every level of 2048 clusters or more in parallel ranges and
    merges them; the near and far pairs still partition all N^2 pairs, and
    with symmetric_far every verdict has its mirror."""
    nodes, tris = inputs.bumpy_ellipsoid(59)
    n = tris.shape[0]
    for sym in (0, 1):
        st = bemfmm.plan_stats_host(nodes, tris, 16000.0, params=bemfmm.default_params(trunc_factor=8.0,
                                                                                           symmetric_far=sym))
        assert st["leaf_level"] >= 6, st
        assert st["near_nnz"] + st["far_pairs"] == n * n
        if sym:
            assert st["asymmetric_pairs"] == 0 and st["asymmetric_near_pairs"] == 0, st


def test_plan_on_ragged_head_like_surface(lib):
    nodes, tris = inputs.bumpy_ellipsoid(13)      # 3380 triangles, uneven sizes
    n = tris.shape[0]
    st = bemfmm.plan_stats_host(nodes, tris, 3000.0)
    assert st["near_nnz"] + st["far_pairs"] == n * n


def test_direct_mode_plan_is_dense(lib):
    nodes, tris = inputs.icosphere(2, 0.1)
    p = bemfmm.default_params(mode=bemfmm.MODE_DIRECT)
    st = bemfmm.plan_stats_host(nodes, tris, 1000.0, params=p)
    assert st["near_nnz"] == tris.shape[0] ** 2 and st["far_pairs"] == 0 and st["levels"] == 0


def test_low_frequency_falls_back_to_near_field(lib):
    """At low k the Hankel growth bound (FP32 stability) rejects far pairs."""
    nodes, tris = inputs.icosphere(4, 0.1)
    hi = bemfmm.plan_stats_host(nodes, tris, 4000.0)
    lo = bemfmm.plan_stats_host(nodes, tris, 50.0)
    assert lo["far_pairs"] < hi["far_pairs"]


def test_bad_arguments_are_rejected(lib):
    nodes, tris = inputs.icosphere(1, 0.1)
    bad = tris.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(bemfmm.BemError):
        bemfmm.plan_stats_host(nodes, bad, 1000.0)
    deg = tris.copy()
    deg[0, 1] = deg[0, 0]
    with pytest.raises(bemfmm.BemError):
        bemfmm.plan_stats_host(nodes, deg, 1000.0)


def test_admittance_loss_autograd_convention():
    """bemfmm.admittance_loss hands the library's gradient (dL/dRe Y +
    i dL/dIm Y) to torch.autograd: with a stand-in mesh whose loss is
    sum |Y - Y0|^2 (gradient 2 (Y - Y0) in that convention), Y.grad equals
    what torch's own autograd gives for the same function, also through a
    chain rule factor."""
    torch = pytest.importorskip("torch")
    Y0 = np.array([0.3 + 0.1j, -0.2 + 0.5j, 0.05 - 0.4j])

    class FakeMesh:
        def admittance_gradient(self, freq, sources, y, points, tol, c, rho):
            return float(np.sum(np.abs(y - Y0) ** 2)), 2.0 * (y - Y0), None, None, {"converged": True}

    y = np.array([1.0 - 0.5j, 0.25 + 0.75j, -0.6 + 0.1j])
    Y = torch.tensor(y, dtype=torch.complex128, requires_grad=True)
    L = 3.0 * bemfmm.admittance_loss(FakeMesh(), Y, 1000.0, [], np.zeros((1, 3)))
    L.backward()
    Y2 = torch.tensor(y, dtype=torch.complex128, requires_grad=True)
    L2 = 3.0 * ((Y2 - torch.tensor(Y0)).abs() ** 2).sum()
    L2.backward()
    assert abs(L.item() - L2.item()) < 1e-12
    assert torch.allclose(Y.grad, Y2.grad, atol=1e-12)


def _tet_volume(nodes, tris):
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def test_mesh_check_closed_outward_surfaces(lib):
    """Signed volume against the sum of signed tetrahedra a.(b x c)/6 (the same
    divergence-theorem integral written per vertex triple), no open or
    inconsistently wound edges; the duct's volume is its box's."""
    for nodes, tris in (inputs.icosphere(3, 0.1), inputs.bumpy_ellipsoid(10)):
        r = bemfmm.mesh_check_host(nodes, tris)
        assert r["open_edges"] == 0 and r["misoriented_edges"] == 0
        assert abs(r["volume"] - _tet_volume(nodes, tris)) < 1e-12 * abs(r["volume"])
        assert r["volume"] > 0
    nodes, tris = inputs.duct(0.6, 0.2, 0.1)
    r = bemfmm.mesh_check_host(nodes, tris)
    assert abs(r["volume"] - 0.6 * 0.2 * 0.2) < 1e-12 and r["open_edges"] == 0 and r["misoriented_edges"] == 0


def test_mesh_check_finds_reversed_flipped_and_open(lib):
    nodes, tris = inputs.icosphere(2, 0.1)
    v = bemfmm.mesh_check_host(nodes, tris)["volume"]
    rev = bemfmm.mesh_check_host(nodes, tris[:, [0, 2, 1]])
    assert abs(rev["volume"] + v) < 1e-15 and rev["misoriented_edges"] == 0
    one = tris.copy()
    one[5] = one[5][[0, 2, 1]]
    assert bemfmm.mesh_check_host(nodes, one)["misoriented_edges"] == 3
    assert bemfmm.mesh_check_host(nodes, tris[1:])["open_edges"] == 3


def test_mesh_create_orientation_check_rejects_before_device_work(lib):
    """check_orientation = 1: an inward-wound or inconsistent mesh is an
    argument error raised on the host (this runs without a GPU)."""
    nodes, tris = inputs.icosphere(2, 0.1)
    for bad in (tris[:, [0, 2, 1]], np.concatenate([tris[:5], tris[5:6, [0, 2, 1]], tris[6:]])):
        with pytest.raises(bemfmm.BemError, match="orientation check"):
            bemfmm.Mesh(nodes, bad, check_orientation=1)
    with pytest.raises(bemfmm.BemError):
        bemfmm.Mesh(nodes, tris, check_orientation=2)


def test_plan_lists_symmetric_where_the_verdicts_must_agree(lib):
    """The transposed product reads the lists backwards.  A pair's near/far
    verdict can differ by direction only through the source cluster's
    largest element area in the far test: on a mesh of equal elements (the
    duct's squares) and in direct mode (no far pairs) every list entry has
    its mirror."""
    nodes, tris = inputs.duct(3.4, 0.2, 0.05)
    st = bemfmm.plan_stats_host(nodes, tris, 240.0)
    assert st["levels"] >= 1 and st["asymmetric_pairs"] == 0
    nodes, tris = inputs.bumpy_ellipsoid(10)
    st = bemfmm.plan_stats_host(nodes, tris, 3000.0, params=bemfmm.default_params(mode=bemfmm.MODE_DIRECT))
    assert st["asymmetric_pairs"] == 0 and st["near_nnz"] == tris.shape[0] ** 2


@pytest.mark.parametrize("mesh,freq", [("ico5", 4000.0), ("head20", 5000.0)])
def test_symmetric_far_test_gives_mirrored_lists(lib, mesh, freq):
    """symmetric_far = 1 bounds r~ with the larger of the two clusters'
    element areas: every list entry then has its mirror (the transposed
    product is then the exact transpose), the lists still partition all
    pairs, and only pairs move from the far to the near field."""
    nodes, tris = inputs.icosphere(5, 0.1) if mesh == "ico5" else inputs.bumpy_ellipsoid(20)
    n = tris.shape[0]
    a = bemfmm.plan_stats_host(nodes, tris, freq)
    b = bemfmm.plan_stats_host(nodes, tris, freq, params=bemfmm.default_params(symmetric_far=1))
    assert a["asymmetric_pairs"] > 0 and b["asymmetric_pairs"] == 0
    assert 0 <= a["asymmetric_near_pairs"] <= a["asymmetric_pairs"] and b["asymmetric_near_pairs"] == 0
    assert b["near_nnz"] + b["far_pairs"] == n * n
    assert a["near_nnz"] <= b["near_nnz"] <= 1.5 * a["near_nnz"], (a["near_nnz"], b["near_nnz"])


def _golden_thresholds():
    path = os.path.join(ROOT, "tests", "golden", "order_thresholds.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            tol, m, _, R = line.split()
            rows.append((float(tol), int(m), float(R)))
    return rows


@pytest.mark.parametrize("tol", [1e-3, 1e-6])
def test_library_order_thresholds_match_hand_derived_values(lib, tol):
    """The library's order thresholds (its own Golub-Welsch / order code,
    independent of the oracle's) against the values derived by hand from
    the three a-priori estimates of Sec. 3.1.4 (tests/golden/order_thresholds.txt).
    The oracle is pinned to the same file, so a misreading both shared would
    fail here.  R_1 at 1e-3 is also the library's far-field bound."""
    nodes, tris = inputs.icosphere(2, 0.1)
    p = bemfmm.default_params(quad_tol=tol)
    st = bemfmm.plan_stats_host(nodes, tris, 1000.0, params=p)
    R = st["order_R"]
    assert R[0] == 1.3                    # the subdivision bound of Sec. 3.1.3
    for t, m, Rm in _golden_thresholds():
        if t == tol:
            assert abs(R[m] - Rm) < 2e-6 * Rm, (tol, m, R[m], Rm)


def test_near_quadrature_counts_cover_the_near_field(lib):
    """The near-field work counts (rules of Sec. 3.1 per near pair) add up
    to the near pairs; every element's self term is heavy (Duffy + edge
    rule: 132 kernel evaluations); light entries take 1, 4 or 9 points."""
    nodes, tris = inputs.icosphere(4, 0.1)
    n = tris.shape[0]
    st = bemfmm.plan_stats_host(nodes, tris, 2000.0)
    assert st["near_light_entries"] + st["near_heavy_entries"] == st["near_nnz"]
    assert st["near_heavy_entries"] >= n
    assert st["near_heavy_points"] >= 132 * n
    assert st["near_light_entries"] <= st["near_light_points"] <= 9 * st["near_light_entries"]
    assert st["near_quad_points"] == st["near_light_points"] + st["near_heavy_points"]


@pytest.mark.parametrize("mesh", ["ico4", "head22"])
def test_field_point_plan_partitions_point_element_pairs(lib, mesh):
    """The field-point plan of the FMM evaluation (points clustered on the
    element tree's box grid, far pairs by the element lists' test with the
    points as targets): every point-element pair is either summed directly
    or taken through the expansions, exactly once; distant points go through
    the expansions at coarse levels, points near the surface mostly stay
    near; in direct mode everything is near; a point 2^20 leaf boxes away is
    refused."""
    nodes, tris = inputs.icosphere(4, 0.1) if mesh == "ico4" else inputs.bumpy_ellipsoid(22)
    n = tris.shape[0]
    sets = {"near": inputs.fibonacci_sphere(700, 0.105), "mid": inputs.fibonacci_sphere(900, 0.3),
            "far": inputs.fibonacci_sphere(1500, 1.0)}
    frac = {}
    for name, pts in sets.items():
        st = bemfmm.field_plan_stats_host(nodes, tris, pts, 2000.0)
        m = pts.shape[0]
        assert st["near_pairs"] + st["far_pairs"] == m * n, (name, st)
        assert sum(st["n_point_clusters"]) > 0 or st["far_pairs"] == 0
        assert all(L >= 8 for L in st["L"])
        frac[name] = st["near_pairs"] / (m * n)
    assert frac["far"] == 0.0 and frac["mid"] < 0.01 and frac["near"] > 0.05, frac
    allp = np.vstack(list(sets.values()))
    st = bemfmm.field_plan_stats_host(nodes, tris, allp, 2000.0, params=bemfmm.default_params(mode=bemfmm.MODE_DIRECT))
    assert st["far_pairs"] == 0 and st["near_pairs"] == allp.shape[0] * n
    with pytest.raises(bemfmm.BemError):
        bemfmm.field_plan_stats_host(nodes, tris, np.array([[1e6, 0.0, 0.0]]), 2000.0)
