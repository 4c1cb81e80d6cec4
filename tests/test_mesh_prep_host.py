"""The library's own host-side mesh preparation (mesh_inspect: no device needed) against the
oracle's metrics: dual volumes, the edge list, the edge normals S_ij and the boundary nodal
normals S_i^b, on triangle, hybrid triangle/quadrangle and axisymmetric meshes.  These are the
metrics every kernel consumes; agreement to rounding pins step a0 of the path on the CPU."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


@pytest.fixture(scope="module")
def avip():
    from paper_2201_01291_gb300 import build
    build.build()
    from paper_2201_01291_gb300 import avip as A
    A.load()
    return A


CASES = {
    "triangles": lambda: W.config_small(nx=23, ny=19, seed=5),
    "needle": lambda: W.plates_problem(41, 61, 1e-2, 1.5e-2, 2e4, seed=2, needle_len=2e-3),
    "hybrid": lambda: W.hybrid_plates_problem(21, 17, 1e-2, 0.8e-2, 5e3, seed=3, quad_fraction=0.5),
    "quadrangles": lambda: W.hybrid_plates_problem(15, 13, 1e-2, 1e-2, 5e3, seed=7, quad_fraction=1.0),
    "axisymmetric": lambda: W.axisym_problem(25, 19, 1e-2, 0.8e-2, 1e4, seed=1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_metrics_match_the_oracle(avip, case):
    p = CASES[case]()
    o = O.Oracle(p)
    geom = avip.GEOM_AXISYMMETRIC if getattr(p, "axisymmetric", False) else avip.GEOM_PLANAR
    rc, m = avip.mesh_inspect(p.xy, p.tris, getattr(p, "quads", None), p.node_bc, p.phi_D, geom)
    assert rc == avip.AVIP_OK
    assert m["n_cells"] == p.n_cells
    np.testing.assert_allclose(m["vol"], o.V_node, rtol=1e-13)
    order = np.lexsort((o.edges[:, 1], o.edges[:, 0]))
    np.testing.assert_array_equal(m["edges"], o.edges[order])
    scale = np.abs(o.S_edge).max()
    np.testing.assert_allclose(m["S_edge"], o.S_edge[order], rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(m["S_b"], o.S_b, rtol=0, atol=1e-13 * np.abs(o.S_b).max())
    # structural nonzeros: every pair of vertices sharing a cell, plus the diagonal
    pairs = set()
    for cells in (np.asarray(p.tris).reshape(-1, 3), np.asarray(getattr(p, "quads", None) if getattr(p, "quads", None) is not None else np.zeros((0, 4), int))):
        for c in cells:
            for a in c:
                for b in c:
                    pairs.add((int(a), int(b)))
    assert m["nnz"] == len(pairs)


def test_inspect_rejects_bad_meshes(avip):
    p = W.config_small(nx=9, ny=9)
    bad = p.tris.copy()
    bad[0, 0] = p.n_nodes
    rc, _ = avip.mesh_inspect(p.xy, bad, None, p.node_bc, p.phi_D)
    assert rc == avip.AVIP_EINVAL
    assert "index" in avip.load().avip_inspect_error().decode()
