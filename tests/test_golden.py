"""The integer structure of the discretisation against tests/golden/discretisation_counts.txt
(written by tests/golden/make_golden.py from the oracle alone; Sec. 2.2, Eq. 1.4, Eq. imp,
Eq. 3.1, Sec. 3.2). On CPU: the oracle's brute-force enumeration and closed forms reproduce every
entry, and the closed forms agree with the enumeration on the small meshes. On the GPU: the CUDA
mesh, subdomain and coarse builders give the same counts at the workload sizes."""
import os

import pytest

from oracle.mesh import KuhnMesh, count_all_edges, count_interior_edges, count_closed_box_edges
from oracle import dd

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "discretisation_counts.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = int(v)
    return vals


def test_small_meshes_by_enumeration():
    g = _golden()
    for n in (1, 2, 3, 4, 6):
        m, mi = KuhnMesh(n), KuhnMesh(n, "imp")
        assert g[f"edges_{n}"] == m.edges.shape[0] == count_all_edges(n)
        assert g[f"dofs_pec_{n}"] == m.n_dof == count_interior_edges(n)
        assert g[f"dofs_imp_{n}"] == mi.n_dof == count_all_edges(n)


def test_matrix_pattern_by_pair_count():
    """nnz of K and M = DOF pairs sharing a tetrahedron, counted as a set (not by assembly)."""
    g = _golden()
    for n in (1, 2, 3, 4, 6):
        m = KuhnMesh(n)
        pairs = set()
        for row in m.tet2dof:
            d = [int(x) for x in row if x >= 0]
            pairs.update((a, b) for a in d for b in d)
        assert g[f"nnz_pec_{n}"] == len(pairs)


def test_large_meshes_and_subdomains_by_closed_forms():
    g = _golden()
    for n in (10, 12, 40, 60):
        assert g[f"dofs_pec_{n}"] == count_interior_edges(n)
        assert g[f"dofs_imp_{n}"] == count_all_edges(n)
    for n, core, ov in ((10, 5, 1), (40, 5, 1), (60, 5, 1)):
        boxes = dd.subdomain_boxes(n, core, ov)
        sizes = [count_interior_edges(*(hi - lo).tolist()) for lo, hi in boxes]
        tag = f"{n}_{core}_{ov}"
        assert g[f"sub_count_{tag}"] == len(boxes)
        assert (g[f"sub_min_pec_{tag}"], g[f"sub_max_pec_{tag}"]) == (min(sizes), max(sizes))
        assert g[f"sub_sum_pec_{tag}"] == sum(sizes)
        assert g[f"sub_sum_imp_{tag}"] == sum(count_closed_box_edges(*(hi - lo).tolist()) for lo, hi in boxes)
    for m in (3, 5, 10, 12):
        assert g[f"coarse_dofs_pec_{m}"] == count_interior_edges(m)


@pytest.mark.gpu
def test_cuda_assembly_pattern_matches():
    mx = pytest.importorskip("paper_1711_03789_gb300")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = _golden()
    for n in (2, 3, 4, 6):
        with mx.Problem(n, 2.0, 1.0, 1.0, n, 0, 0, mx.MX_PLAIN_FP64) as P:
            assert P.info()["nnz"] == g[f"nnz_pec_{n}"]


@pytest.mark.gpu
@pytest.mark.parametrize("n,cm", [(10, 5), (40, 10), (60, 12)])
def test_cuda_builders_match(n, cm):
    mx = pytest.importorskip("paper_1711_03789_gb300")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = _golden()
    tag = f"{n}_5_1"
    with mx.Problem(n, 4.0, 0.0, 4.0, 5, 1, cm, mx.MX_MIXED) as P:
        info = P.info()
        assert info["n_dof"] == g[f"dofs_pec_{n}"]
        assert info["n_sub"] == g[f"sub_count_{tag}"]
        assert info["sum_local"] == g[f"sub_sum_pec_{tag}"]
        assert info["max_local"] == g[f"sub_max_pec_{tag}"]
        assert info["n_coarse"] == g[f"coarse_dofs_pec_{cm}"]
    with mx.Problem(n, 4.0, 0.0, 4.0, 5, 1, 0, mx.MX_MIXED, bc=mx.MX_BC_IMPEDANCE) as P:
        info = P.info()
        assert info["n_dof"] == g[f"dofs_imp_{n}"]
        assert info["sum_local"] == g[f"sub_sum_imp_{tag}"]
