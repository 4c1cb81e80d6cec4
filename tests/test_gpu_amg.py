"""Parity of the AMG-preconditioned conjugate-gradient solve (solver kind 8: smoothed
aggregation hierarchy built once per mesh, one V-cycle per CG iteration) with the FP64
oracle's direct solve and with the Jacobi-PCG path.  Tolerances as for the other FP64 paths:
norm-wise 1e-12 on a lone Poisson solve at rtol 1e-14, 1e-10 on phi and densities after steps."""
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


@pytest.mark.parametrize("nx,ny", [(13, 11), (40, 33), (161, 127)])
def test_amg_poisson_parity(avip, nx, ny):
    """Ragged node counts, one to four levels below the finest."""
    p = W.config_small(nx=nx, ny=ny, seed=nx * ny)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=8)
    assert m.info["pcg_kind"] == 8
    it, rr = m.poisson_solve()
    assert rr <= 1e-14
    assert normwise(m.phi(), phi_ref) <= 1e-12
    m.close()


def test_amg_needs_far_fewer_iterations(avip):
    """On a 301 x 301 mesh the V-cycle preconditioner cuts the CG iteration count by more than
    five times against Jacobi (same rtol, same answer)."""
    p = W.plates_problem(301, 301, 1e-2, 1e-2, 1e4, seed=6, field_dependent=True, source=W.SRC_TOWNSEND)
    ja = avip.Mesh(p, rtol=1e-12, pcg_kind=1)
    am = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    it_j, _ = ja.poisson_solve()
    it_a, rr = am.poisson_solve()
    assert rr <= 1e-12
    assert it_a * 5 < it_j, (it_a, it_j)
    assert normwise(am.phi(), ja.phi()) <= 1e-10
    ja.close()
    am.close()


def test_amg_steps_parity_pin_plane_small(avip):
    """Needle anode, field-dependent mobility, Townsend ionisation: 20 steps against the oracle."""
    p = W.plates_problem(41, 81, 1e-2, 2e-2, 2e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND,
                         needle_len=2e-3)
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(20)
    m = avip.Mesh(p, rtol=1e-13, pcg_kind=8)
    st = m.run(20)
    assert st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    m.close()


def test_amg_auto_for_large_meshes_and_steps(avip):
    """Above the cluster size the automatic choice is the AMG solver; 10 steps of a
    51,000-node mesh with three species against the oracle."""
    p = W.plates_problem(255, 201, 1e-2, 0.8e-2, 2e4, seed=12, field_dependent=True,
                         source=W.SRC_TOWNSEND_ATTACH, n_species=3)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(10)
    m = avip.Mesh(p, rtol=1e-13)
    assert m.info["pcg_kind"] == 8
    st = m.run(10)
    assert st["status"] == 0
    for s in range(3):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    m.close()


def test_amg_graph_replay_and_checkpoint_bitwise(avip):
    p = W.plates_problem(121, 97, 1e-2, 0.8e-2, 2e4, seed=3, field_dependent=True, source=W.SRC_TOWNSEND)
    a = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    b = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    a.run(8)
    for _ in range(8):
        b.step()
    for s in range(2):
        assert np.array_equal(a.density(s), b.density(s))
    st = a.state()
    a.run(4)
    b.set_state(st)
    b.run(4)
    assert np.array_equal(a.density(0), b.density(0))
    a.close()
    b.close()


def test_amg_large_mesh_poisson(avip):
    """A quarter-million-node mesh with the needle: the solve against the oracle's direct
    solve at rtol 1e-13."""
    p = W.plates_problem(401, 631, 1e-2, 1.6e-2, 2e4, seed=9, needle_len=2e-3)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-13, pcg_kind=8)
    it, rr = m.poisson_solve()
    assert rr <= 1e-13 and 0 < it < 200
    assert normwise(m.phi(), phi_ref) <= 1e-10
    m.close()


def test_mixed_amg_poisson_and_auto_choice(avip):
    """Mixed precision with the AMG preconditioner (kind 10): FP32 inner CG and V-cycle, FP64
    refinement to rtol 1e-12, against the oracle's direct solve; automatic above the cluster
    size."""
    p = W.plates_problem(255, 201, 1e-2, 0.8e-2, 2e4, seed=12, field_dependent=True, source=W.SRC_TOWNSEND)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-12)
    assert m.info["pcg_kind"] == 10
    it, rr = m.poisson_solve()
    assert rr <= 1e-12
    assert normwise(m.phi(), phi_ref) <= 1e-10
    m.close()


def test_mixed_amg_steps_within_1e6(avip):
    """FP32 gradients, fluxes and inner solve: 50 steps of the reduced pin-plane case within
    1e-6 of the FP64 oracle."""
    p = W.plates_problem(41, 81, 1e-2, 2e-2, 2e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND,
                         needle_len=2e-3)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(50)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10, pcg_kind=10)
    assert m.info["pcg_kind"] == 10
    st = m.run(50)
    assert st["status"] == 0
    errs = [normwise(m.density(s), n_ref[s]) for s in range(2)] + [normwise(m.phi(), phi_ref)]
    print("mixed AMG 50-step norm-wise errors (n_e, n_+, phi):", errs)
    assert max(errs) <= 1e-6
    m.close()


def test_predictor_cuts_iterations_and_resumes_bitwise(avip):
    """The initial guess extrapolated from the last potentials: fewer CG iterations than the
    plain warm start (history cleared through the state before every step), the same answer
    within the solve tolerance, and the history travels with the checkpoint."""
    p = W.plates_problem(161, 161, 1e-2, 1e-2, 2e4, seed=4, field_dependent=True, source=W.SRC_TOWNSEND)
    m = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    m.run(20)
    snap = m.state()
    assert snap[-1] == 3.0
    it_pred = m.run(10)["pcg_iters_total"]
    cold = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    cold.set_state(snap)
    it_cold = 0
    for _ in range(10):
        s = cold.state()
        s[-1] = 0.0
        cold.set_state(s)
        it_cold += cold.run(1)["pcg_iters_total"]
    assert it_pred < it_cold, (it_pred, it_cold)
    for s in range(2):
        assert normwise(m.density(s), cold.density(s)) <= 1e-10
    resumed = avip.Mesh(p, rtol=1e-12, pcg_kind=8)
    resumed.set_state(snap)
    resumed.run(10)
    np.testing.assert_array_equal(resumed.state(), m.state())
    for x in (m, cold, resumed):
        x.close()


@pytest.mark.parametrize("csize", [2, 4, 8, 16])
def test_amg_cluster_solve_every_cluster_size(avip, csize):
    """The AMG solve on one thread-block cluster (kind 11) with 2, 4, 8 and 16 CTAs: the same
    potential as the oracle's direct solve (1e-12 at rtol 1e-14) and, after 8 steps, the same
    densities as the whole-GPU AMG solve (1e-11: both converge to rtol 1e-14)."""
    p = W.plates_problem(97, 113, 1e-2, 1.2e-2, 1.5e4, seed=61, field_dependent=True, source=W.SRC_TOWNSEND)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=11, cluster_size=csize)
    assert m.info["pcg_kind"] == 11 and m.info["pcg_blocks"] == csize
    m.poisson_solve()
    assert normwise(m.phi(), phi_ref) <= 1e-12
    g = avip.Mesh(p, rtol=1e-14, pcg_kind=8)
    m.run(8)
    g.run(8)
    for s in range(2):
        assert normwise(m.density(s), g.density(s)) <= 1e-11
    m.close()
    g.close()
