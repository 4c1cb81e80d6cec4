"""Parity of the GPU path on quadrangle and hybrid (triangle + quadrangle) meshes with the FP64
oracle: the Poisson solve with every planar solver kind, explicit steps with the LLW and SG
fluxes, field-dependent mobility and Townsend sources, the time step over four-vertex cells, a
large quadrangle mesh on the AMG solver, mixed precision, and a hybrid instance inside a batch.
Tolerances: norm-wise 1e-12 on a lone solve at rtol 1e-14, 1e-10 on phi and densities after
steps (FP64), 1e-6 for mixed precision."""
import numpy as np
import pytest

import avip_oracle as O
from helpers import normwise
from paper_2201_01291_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def avip():
    from paper_2201_01291_gb300 import build
    build.build()
    from paper_2201_01291_gb300 import avip as A
    A.load()
    return A


def hybrid(nx, ny, frac, seed, **kw):
    kw.setdefault("field_dependent", True)
    kw.setdefault("source", W.SRC_TOWNSEND)
    return W.hybrid_plates_problem(nx, ny, 1e-2, 0.9e-2, 2.5e4, seed=seed, quad_fraction=frac, **kw)


def test_hybrid_mesh_info(avip):
    p = hybrid(33, 29, 0.5, seed=2)
    m = avip.Mesh(p)
    o = O.Oracle(p)
    assert m.info["n_nodes"] == p.n_nodes
    assert m.info["n_cells"] == p.tris.shape[0] + p.quads.shape[0]
    assert m.info["n_edges"] == o.edges.shape[0]
    m.close()


@pytest.mark.parametrize("kind", [1, 2, 5, 8, 11])
def test_hybrid_poisson_parity(avip, kind):
    p = hybrid(33, 29, 0.5, seed=kind)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=kind)
    assert m.info["pcg_kind"] == kind
    it, rr = m.poisson_solve()
    assert rr <= 1e-14
    assert normwise(m.phi(), phi_ref) <= 1e-12
    m.close()


def test_hybrid_single_step_dt(avip):
    """One step: the automatic time step (cell averages over three or four vertices, shortest
    side) and the densities."""
    p = hybrid(21, 19, 0.5, seed=3)
    o = O.Oracle(p)
    n1, info = o.step(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    dt = m.step()
    assert abs(dt - info["dt"]) <= 1e-12 * info["dt"]
    for s in range(2):
        assert normwise(m.density(s), n1[s]) <= TOL
    m.close()


@pytest.mark.parametrize("frac,scheme,species", [(1.0, W.FLUX_LLW, 2), (0.5, W.FLUX_LLW, 3),
                                                 (0.5, W.FLUX_SG, 2), (0.3, W.FLUX_SG, 3)])
def test_hybrid_steps_parity(avip, frac, scheme, species):
    src = W.SRC_TOWNSEND_ATTACH if species == 3 else W.SRC_TOWNSEND
    p = hybrid(37, 31, frac, seed=11, source=src, n_species=species)
    p.opts.scheme = scheme
    nsteps = 15
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, rtol=1e-13)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(species):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n_ref)
    assert abs(st["charge"] - o.charge(n_ref)) <= 1e-10 * scale
    m.close()


def test_quadrangle_mesh_amg_steps(avip):
    """A 36,000-node quadrangle mesh: the automatic AMG-CG solver and 8 steps against the
    oracle."""
    p = hybrid(201, 181, 1.0, seed=5)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(8)
    m = avip.Mesh(p, rtol=1e-13)
    assert m.info["pcg_kind"] == 8
    st = m.run(8)
    assert st["status"] == 0
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    m.close()


def test_hybrid_mixed_within_1e6(avip):
    p = hybrid(41, 37, 0.5, seed=8)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(40)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10)
    st = m.run(40)
    assert st["status"] == 0
    errs = [normwise(m.density(s), n_ref[s]) for s in range(2)] + [normwise(m.phi(), phi_ref)]
    assert max(errs) <= 1e-6, errs
    m.close()


def test_hybrid_instance_in_batch_equals_alone(avip):
    ps = [W.config_small(nx=25, ny=23, seed=1), hybrid(29, 27, 0.5, seed=2), hybrid(23, 31, 1.0, seed=3)]
    nsteps = 6
    meshes = [avip.Mesh(p, rtol=1e-13, pcg_kind=5) for p in ps]
    b = avip.Batch(meshes)
    b.run(nsteps)
    for k, p in enumerate(ps):
        alone = avip.Mesh(p, rtol=1e-13, pcg_kind=5)
        alone.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), alone.density(s)) <= 1e-12, (k, s)
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), n_ref[s]) <= TOL, (k, s)
        alone.close()
    b.close()
