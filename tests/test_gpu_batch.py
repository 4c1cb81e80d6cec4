"""Batched instances: every instance gives the same result alone and inside a batch of
uneven sizes and species counts, and matches the FP64 oracle."""
import numpy as np
import pytest

import avip_oracle as O
from helpers import normwise
from paper_2201_01291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def avip():
    from paper_2201_01291_gb300 import build
    build.build()
    from paper_2201_01291_gb300 import avip as A
    A.load()
    return A


def _instances():
    ps = W.random_instances(6, seed=4, t_min=500, t_max=6000)
    return ps


@pytest.mark.parametrize("cluster_size", [16, 8, 0])
def test_batch_equals_alone(avip, cluster_size):
    ps = _instances()
    nsteps = 8
    batch_meshes = [avip.Mesh(p, rtol=1e-13, pcg_kind=5) for p in ps]  # the shared-memory Jacobi solver
    b = avip.Batch(batch_meshes, cluster_size=cluster_size)
    # the drift-diffusion block: tuned with cluster_size 0, else 256; set to 128 for 8 CTAs so
    # that both partitions are exercised
    assert b.info["dd_threads"] in ((128, 256) if cluster_size == 0 else (256,))
    if cluster_size == 8:
        assert avip.batch_set_dd_threads(b.b, 128) == avip.AVIP_OK
        assert avip.batch_set_dd_threads(b.b, 96) == avip.AVIP_EINVAL
        assert avip.batch_info(b.b)["dd_threads"] == 128
    st = b.run(nsteps)
    assert all(s["steps"] == nsteps for s in st)
    C = b.info["cluster_size"]
    for k, p in enumerate(ps):
        alone = avip.Mesh(p, rtol=1e-13, pcg_kind=5)
        alone.run(nsteps)
        for s in range(len(p.species)):
            a = alone.density(s)
            m = batch_meshes[k].density(s)
            assert normwise(m, a) <= 1e-12, (k, s, C)
        assert normwise(batch_meshes[k].phi(), alone.phi()) <= 1e-12
        alone.close()
    b.close()


def test_batch_matches_oracle(avip):
    ps = _instances()[:3]
    nsteps = 6
    meshes = [avip.Mesh(p, rtol=1e-13) for p in ps]
    b = avip.Batch(meshes)
    b.run(nsteps)
    for k, p in enumerate(ps):
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), n_ref[s]) <= 1e-10, (k, s)
        assert normwise(meshes[k].phi(), phi_ref) <= 1e-10
    b.close()


def test_mixed_batch_equals_alone_and_oracle(avip):
    """Mixed-precision instances (FP32 inner CG + FP64 refinement inside each cluster) give the
    same result in a batch as alone, and stay within 1e-6 of the FP64 oracle."""
    ps = _instances()[:4]
    nsteps = 6
    meshes = [avip.Mesh(p, rtol=1e-11, precision=avip.PREC_MIXED, pcg_kind=6) for p in ps]
    b = avip.Batch(meshes, cluster_size=16)   # the cluster size the single-instance plan picks
    b.run(nsteps)
    for k, p in enumerate(ps):
        alone = avip.Mesh(p, rtol=1e-11, precision=avip.PREC_MIXED, pcg_kind=6)
        assert alone.info["pcg_kind"] == 6
        alone.run(nsteps)
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), alone.density(s)) <= 1e-12
            assert normwise(meshes[k].density(s), n_ref[s]) <= 1e-6
        assert normwise(meshes[k].phi(), phi_ref) <= 1e-6
        alone.close()
    b.close()


def test_batch_with_amg_instances(avip):
    """Instances with an AMG hierarchy (the two above the cluster size, and the mid-size one
    whose own solver is the one-cluster AMG form) are solved inside the batch by the cluster
    form of the AMG-preconditioned CG.  Every instance matches the oracle; against the same instance alone (whole-GPU AMG
    kernel, whose dot products are summed in another order) within 1e-10."""
    ps = [W.plates_problem(181, 151, 1e-2, 0.8e-2, 2e4, seed=51, field_dependent=True, source=W.SRC_TOWNSEND),
          W.plates_problem(35, 29, 1e-2, 0.8e-2, 1.5e4, seed=52, field_dependent=True, source=W.SRC_TOWNSEND),
          W.plates_problem(151, 201, 1e-2, 1.3e-2, 2.2e4, seed=53, field_dependent=True,
                           source=W.SRC_TOWNSEND_ATTACH, n_species=3)]
    nsteps = 5
    meshes = [avip.Mesh(p, rtol=1e-13) for p in ps]
    assert [m.info["pcg_kind"] for m in meshes] == [8, 11, 8]
    b = avip.Batch(meshes, cluster_size=16)
    b.run(nsteps)
    for k, p in enumerate(ps):
        alone = avip.Mesh(p, rtol=1e-13)
        alone.run(nsteps)
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), n_ref[s]) <= 1e-10, (k, s)
            assert normwise(meshes[k].density(s), alone.density(s)) <= 1e-10, (k, s)
        assert normwise(meshes[k].phi(), phi_ref) <= 1e-10
        alone.close()
    b.close()


def test_mixed_batch_with_amg_instances(avip):
    """Mixed-precision instances with an FP32 AMG hierarchy (kind 10) inside a batch: within
    1e-6 of the FP64 oracle, and close to the same instance solved alone by the whole-GPU
    mixed AMG kernel."""
    ps = [W.plates_problem(121, 101, 1e-2, 0.8e-2, 2e4, seed=61, field_dependent=True, source=W.SRC_TOWNSEND),
          W.plates_problem(61, 41, 1e-2, 0.8e-2, 1.5e4, seed=62, field_dependent=True, source=W.SRC_TOWNSEND)]
    nsteps = 5
    meshes = [avip.Mesh(p, rtol=1e-11, precision=avip.PREC_MIXED, pcg_kind=10) for p in ps]
    b = avip.Batch(meshes, cluster_size=16)
    b.run(nsteps)
    for k, p in enumerate(ps):
        alone = avip.Mesh(p, rtol=1e-11, precision=avip.PREC_MIXED, pcg_kind=10)
        alone.run(nsteps)
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(nsteps)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), n_ref[s]) <= 1e-6, (k, s)
            assert normwise(meshes[k].density(s), alone.density(s)) <= 1e-8, (k, s)
        assert normwise(meshes[k].phi(), phi_ref) <= 1e-6
        alone.close()
    b.close()


def test_batch_checkpoint_round_trip(avip):
    """batch_state_get equals the instances' own states concatenated; batch_state_set restores
    them (the batch then repeats its steps bit for bit) and refuses a non-finite entry."""
    ps = _instances()[:4]
    meshes = [avip.Mesh(p, rtol=1e-13, pcg_kind=5) for p in ps]
    b = avip.Batch(meshes, cluster_size=16)
    b.run(2)
    snap = b.state()
    np.testing.assert_array_equal(snap, np.concatenate([m.state() for m in meshes]))
    b.run(3)
    after = b.state()
    bad = snap.copy()
    bad[5] = np.inf
    assert avip.batch_state_set(b.b, bad) == avip.AVIP_ENAN
    np.testing.assert_array_equal(b.state(), after)  # nothing installed
    b.set_state(snap)
    b.run(3)
    np.testing.assert_array_equal(b.state(), after)
    b.close()
