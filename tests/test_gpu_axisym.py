"""Parity of the axisymmetric (x, r) CUDA path (r-weighted metrics, BiCGStab on the
non-symmetric Poisson matrix) with the FP64 CPU oracle on the same seeded inputs.  Tolerances
as for the planar path: norm-wise 1e-12 on a Poisson solve alone, 1e-10 on phi and densities
after many steps."""
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


@pytest.mark.parametrize("nx,nr", [(9, 7), (33, 17), (61, 45)])
def test_axisym_poisson_parity(avip, nx, nr):
    """Ragged node counts (several 32-row slices plus a tail), nodes on the axis."""
    p = W.axisym_problem(nx, nr, 1e-2, 0.6e-2, 2e4, seed=nx * nr)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    assert m.info["pcg_kind"] == 7
    it, rr = m.poisson_solve()
    assert rr <= 1e-14
    assert normwise(m.phi(), phi_ref) <= 1e-12
    E_ref = -O.nodal_gradient(phi_ref, o.tris, o.S, o.V_tau, o.A_node)
    E = np.stack([m.field(avip.FIELD_EX), m.field(avip.FIELD_EY)], axis=1)
    assert normwise(E, E_ref) <= 1e-11
    assert normwise(m.field(avip.FIELD_VOLUME), o.V_node) <= 1e-14
    m.close()


def test_axisym_single_step_parity(avip):
    p = W.axisym_problem(25, 19, 1e-2, 0.6e-2, 2e4, seed=5)
    o = O.Oracle(p)
    n1, info = o.step(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    dt = m.step()
    assert abs(dt - info["dt"]) <= 1e-12 * info["dt"]
    for s in range(2):
        assert normwise(m.density(s), n1[s]) <= TOL
    assert normwise(m.phi(), info["phi"]) <= TOL
    m.close()


@pytest.mark.parametrize("limiter,beta", [(W.LIM_SWEBY, 1.0), (W.LIM_VANLEER, 1.0)])
def test_axisym_townsend_60_steps_parity(avip, limiter, beta):
    """Field-dependent mobility, Townsend ionisation, outflow closure for electrons."""
    p = W.axisym_problem(41, 27, 1e-2, 0.6e-2, 2.5e4, seed=11, field_dependent=True, source=W.SRC_TOWNSEND)
    p.opts.limiter, p.opts.beta = limiter, beta
    p.species[0].bnd_mode = W.BND_OUTFLOW
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(60)
    m = avip.Mesh(p, rtol=1e-13)
    st = m.run(60)
    assert st["steps"] == 60 and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n_ref)
    assert abs(st["charge"] - o.charge(n_ref)) <= 1e-10 * scale
    m.close()


def test_axisym_three_species_parity(avip):
    p = W.axisym_problem(29, 21, 1e-2, 0.6e-2, 2.5e4, seed=17, field_dependent=True,
                         source=W.SRC_TOWNSEND_ATTACH, n_species=3)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(25)
    m = avip.Mesh(p, rtol=1e-13)
    st = m.run(25)
    assert st["status"] == 0
    for s in range(3):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    m.close()


def test_bicgstab_on_planar_mesh_matches_oracle(avip):
    """BiCGStab (kind 7) also solves the symmetric planar system."""
    p = W.plates_problem(23, 29, 1e-2, 1.2e-2, 2.5e4, seed=9, field_dependent=True, source=W.SRC_TOWNSEND)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(20)
    m = avip.Mesh(p, rtol=1e-13, pcg_kind=7)
    assert m.info["pcg_kind"] == 7
    st = m.run(20)
    assert st["status"] == 0
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    m.close()


def test_axisym_graph_replay_and_checkpoint(avip):
    """Graph replay of many steps equals single steps; state set/get resumes bit for bit."""
    p = W.axisym_problem(21, 17, 1e-2, 0.6e-2, 2e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND)
    a = avip.Mesh(p, rtol=1e-13)
    a.run(12)
    b = avip.Mesh(p, rtol=1e-13)
    for _ in range(12):
        b.step()
    for s in range(2):
        assert np.array_equal(a.density(s), b.density(s))
    st = a.state()
    a.run(5)
    b.set_state(st)
    b.run(5)
    assert np.array_equal(a.density(0), b.density(0))
    a.close()
    b.close()


def test_axisym_large_mesh_sampled(avip):
    """A quarter-million-node axisymmetric mesh: the Poisson solve against the oracle's
    direct solve, and the relative residual reached."""
    p = W.axisym_problem(701, 361, 2.5e-2, 1.25e-2, 3e4, seed=7, sigma=2e-3)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-13)
    it, rr = m.poisson_solve()
    assert rr <= 1e-13 and it > 0
    assert normwise(m.phi(), phi_ref) <= 1e-10
    m.close()


@pytest.mark.parametrize("nx,nr", [(33, 17), (61, 45), (161, 121)])
def test_axisym_amg_bicgstab_poisson_parity(avip, nx, nr):
    """BiCGStab right-preconditioned by the AMG V-cycle (kind 9) on the non-symmetric matrix."""
    p = W.axisym_problem(nx, nr, 1e-2, 0.6e-2, 2e4, seed=nx + nr)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=9)
    assert m.info["pcg_kind"] == 9
    it, rr = m.poisson_solve()
    assert rr <= 1e-14
    assert normwise(m.phi(), phi_ref) <= 1e-12
    m.close()


def test_axisym_amg_cuts_iterations_and_steps_parity(avip):
    """On a 301 x 201 axisymmetric mesh the preconditioned BiCGStab needs far fewer iterations
    than the Jacobi-scaled one at the same rtol; its solve at rtol 1e-13 matches the oracle's
    direct solve; 15 steps with Townsend against the oracle."""
    p = W.axisym_problem(301, 201, 1e-2, 0.6e-2, 2.5e4, seed=21, field_dependent=True, source=W.SRC_TOWNSEND)
    ja = avip.Mesh(p, rtol=1e-12, pcg_kind=7)
    am = avip.Mesh(p, rtol=1e-12)
    assert am.info["pcg_kind"] == 9
    it_j, _ = ja.poisson_solve()
    it_a, rr = am.poisson_solve()
    assert rr <= 1e-12 and it_a * 10 < it_j, (it_a, it_j)
    ja.close()
    am.close()
    o = O.Oracle(p)
    m = avip.Mesh(p, rtol=1e-13)
    m.poisson_solve()
    assert normwise(m.phi(), o.poisson(o.initial_state())) <= 1e-10
    m.close()
    n_ref, phi_ref, _ = o.run(15)
    m = avip.Mesh(p, rtol=1e-13)
    st = m.run(15)
    assert st["status"] == 0
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    m.close()
