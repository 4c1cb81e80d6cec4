"""CPU-side checks of the C ABI: the library builds, loads and exports every function that
include/avip.h declares; host-only entry points behave.  No GPU compute is called."""
import os

import numpy as np
import pytest

from helpers import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_01291_gb300 import build
    build.build()
    from paper_2201_01291_gb300 import avip
    return avip.load()


def test_header_symbols_exported(lib):
    names = header_functions(os.path.join(ROOT, "include", "avip.h"))
    assert "mesh_create" in names and "run_steps" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2201_01291_gb300 import avip
    names = header_functions(os.path.join(ROOT, "include", "avip.h"))
    assert set(names) <= set(avip.exported_symbols())


def test_host_only_entry_points(lib):
    from paper_2201_01291_gb300 import avip
    o = avip.avip_opts_default()
    assert o.cfl == 0.4 and o.rtol == 1e-12 and o.reorder == 1 and o.precision == 0
    assert avip.status_str(avip.AVIP_ENOTCONV).startswith("PCG")
    assert avip.status_str(12345) == "unknown status"
    assert lib.mesh_destroy(None) == 0
    # null handles are rejected before any device work
    assert avip.batch_set_dd_threads(None, 128) == avip.AVIP_EINVAL
    assert avip.photo_stats(None)[0] == avip.AVIP_EINVAL
    assert avip.state_set(None, np.zeros(4)) == avip.AVIP_EINVAL


def test_mesh_validation_on_host(lib):
    """mesh_create rejects bad meshes in host code before any CUDA call (runs without a GPU)."""
    import numpy as np
    from paper_2201_01291_gb300 import avip, workloads as W
    p = W.config_small(nx=9, ny=9)
    o = avip.avip_opts_default()
    bad = p.tris.copy()
    bad[0, 0] = p.n_nodes + 5
    assert avip.mesh_create(p.xy, bad, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "out of range" in avip.last_error()
    deg = p.tris.copy()
    deg[0, 1] = deg[0, 0]
    assert avip.mesh_create(p.xy, deg, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "zero-area" in avip.last_error()
    assert avip.mesh_create(p.xy, p.tris, np.zeros_like(p.node_bc), p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "Dirichlet" in avip.last_error()
    bc = p.node_bc.copy()
    bc[0] = 7
    assert avip.mesh_create(p.xy, p.tris, bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    xy = p.xy.copy()
    xy[4, 0] = np.inf
    assert avip.mesh_create(xy, p.tris, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    o2 = avip.avip_opts_default()
    o2.rtol = -1.0
    assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o2)[0] == avip.AVIP_EINVAL
    # the device-wait limit: default 2 s, 0 allowed (fail at the first wait), negative, NaN or
    # above 60 s rejected before any CUDA call
    assert avip.avip_opts_default().wait_timeout == 2.0
    for bad_limit in (-1.0, float("nan"), 61.0):
        o3 = avip.avip_opts_default()
        o3.wait_timeout = bad_limit
        assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o3)[0] == avip.AVIP_EINVAL
    assert avip.mesh_set_wait_timeout(None, 1.0) == avip.AVIP_EINVAL
    o4 = avip.avip_opts_default()
    o4.cluster_size = 3  # 2, 4, 8, 16 or 0 only
    assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o4)[0] == avip.AVIP_EINVAL


def test_axisymmetric_validation_on_host(lib):
    """Axisymmetric options are checked on the host: negative radius, unknown geometry, and
    solvers that need a symmetric matrix (CG kinds, mixed precision) are rejected."""
    from paper_2201_01291_gb300 import avip, workloads as W
    p = W.axisym_problem(9, 7, 1e-2, 0.5e-2, 1e4, seed=1)
    o = avip.avip_opts_default()
    assert o.geometry == avip.GEOM_PLANAR
    o.geometry = avip.GEOM_AXISYMMETRIC
    xy = p.xy.copy()
    xy[3, 1] = -1e-3
    assert avip.mesh_create(xy, p.tris, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "negative radius" in avip.last_error()
    for kind, prec in ((2, avip.PREC_FP64), (1, avip.PREC_FP64), (0, avip.PREC_MIXED)):
        o2 = avip.avip_opts_default()
        o2.geometry, o2.pcg_kind, o2.precision = avip.GEOM_AXISYMMETRIC, kind, prec
        assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o2)[0] == avip.AVIP_EINVAL
        assert "BiCGStab" in avip.last_error()
    o3 = avip.avip_opts_default()
    o3.geometry = 5
    assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o3)[0] == avip.AVIP_EINVAL
    assert "geometry" in avip.last_error()


def test_unknown_flux_scheme_rejected_on_host(lib):
    from paper_2201_01291_gb300 import avip, workloads as W
    p = W.config_small(nx=9, ny=9)
    o = avip.avip_opts_default()
    assert o.scheme == avip.FLUX_LLW
    o.scheme = 3
    assert avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL


def test_hybrid_mesh_validation_on_host(lib):
    """mesh_create_hybrid rejects quadrangle indices out of range, zero-area quadrangles, an
    empty cell list and quadrangles in the axisymmetric geometry, in host code."""
    import numpy as np
    from paper_2201_01291_gb300 import avip, workloads as W
    p = W.hybrid_plates_problem(9, 7, 1e-2, 0.8e-2, 5e3, seed=3, quad_fraction=0.5)
    o = avip.avip_opts_default()
    bad = p.quads.copy()
    bad[2, 3] = p.n_nodes
    assert avip.mesh_create_hybrid(p.xy, p.tris, bad, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "quadrangle index" in avip.last_error()
    deg = p.quads.copy()
    deg[0] = [deg[0, 0], deg[0, 1], deg[0, 1], deg[0, 0]]
    assert avip.mesh_create_hybrid(p.xy, p.tris, deg, p.node_bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "quadrangle" in avip.last_error()
    empty = np.zeros((0, 3), np.int32)
    assert avip.mesh_create_hybrid(p.xy, empty, np.zeros((0, 4), np.int32), p.node_bc, p.phi_D,
                                   o)[0] == avip.AVIP_EINVAL
    oa = avip.avip_opts_default()
    oa.geometry = avip.GEOM_AXISYMMETRIC
    assert avip.mesh_create_hybrid(p.xy, p.tris, p.quads, p.node_bc, p.phi_D, oa)[0] == avip.AVIP_EINVAL
    assert "planar" in avip.last_error()


def test_node_bc_values_on_host(lib):
    """node_bc accepts 0, 1 and 2 (a Neumann side's node) and rejects anything else."""
    import numpy as np
    from paper_2201_01291_gb300 import avip, workloads as W
    p = W.config_small(nx=9, ny=9)
    o = avip.avip_opts_default()
    bc = p.node_bc.copy()
    bc[3] = 3
    assert avip.mesh_create(p.xy, p.tris, bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
    assert "node_bc" in avip.last_error()
    bc[3] = -1
    assert avip.mesh_create(p.xy, p.tris, bc, p.phi_D, o)[0] == avip.AVIP_EINVAL
