"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the same seeded
inputs.  Tolerance: norm-wise max relative error <= 1e-10 on phi and every density (FP64),
1e-12 on the time step and the Poisson solution alone."""
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


def run_both(avip, problem, nsteps, rtol=1e-13, **kw):
    o = O.Oracle(problem)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(problem, rtol=rtol, **kw)
    st = m.run(nsteps)
    n_gpu = [m.density(s) for s in range(len(problem.species))]
    return o, m, st, n_ref, phi_ref, dts, n_gpu, m.phi()


@pytest.mark.parametrize("nx,ny", [(13, 11), (17, 17), (40, 33)])
def test_poisson_parity(avip, nx, ny):
    p = W.config_small(nx=nx, ny=ny, seed=nx * ny)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    it, rr = m.poisson_solve()
    assert rr <= 1e-14
    assert normwise(m.phi(), phi_ref) <= 1e-12
    # E from the GPU gradient vs the oracle's nodal gradient of its own phi
    E_ref = -O.nodal_gradient(phi_ref, o.tris, o.S, o.V_tau, o.V_node)
    E = np.stack([m.field(avip.FIELD_EX), m.field(avip.FIELD_EY)], axis=1)
    assert normwise(E, E_ref) <= 1e-11
    assert normwise(m.field(avip.FIELD_VOLUME), o.V_node) <= 1e-14


def test_single_step_parity(avip):
    p = W.config_small(nx=21, ny=19, seed=3)
    o = O.Oracle(p)
    n1, info = o.step(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    dt = m.step()
    assert abs(dt - info["dt"]) <= 1e-12 * info["dt"]
    for s in range(2):
        assert normwise(m.density(s), n1[s]) <= TOL
    assert normwise(m.phi(), info["phi"]) <= TOL


def test_plates65_100_steps_parity(avip):
    """Plain FP64 parallel plates: 65 x 65 nodes (8192 triangles), 100 explicit steps."""
    p = W.config_plates_65()
    o, m, st, n_ref, phi_ref, dts, n_gpu, phi = run_both(avip, p, 100)
    assert st["steps"] == 100 and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(2):
        assert normwise(n_gpu[s], n_ref[s]) <= TOL, s
    assert normwise(phi, phi_ref) <= TOL
    # charge after the run
    assert abs(st["charge"] - o.charge(n_ref)) <= 1e-10 * sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n_ref)


@pytest.mark.parametrize("limiter,beta", [(W.LIM_SWEBY, 1.5), (W.LIM_VANLEER, 1.0)])
def test_source_field_dependent_parity(avip, limiter, beta):
    """Townsend ionisation, local-field mobility, outflow closure, other limiters, ragged N."""
    p = W.plates_problem(23, 29, 1e-2, 1.2e-2, 2.5e4, seed=9, field_dependent=True, source=W.SRC_TOWNSEND)
    p.opts.limiter, p.opts.beta = limiter, beta
    p.species[0].bnd_mode = W.BND_OUTFLOW
    _, _, st, n_ref, phi_ref, _, n_gpu, phi = run_both(avip, p, 30)
    for s in range(2):
        assert normwise(n_gpu[s], n_ref[s]) <= TOL
    assert normwise(phi, phi_ref) <= TOL


def test_three_species_attachment_parity(avip):
    p = W.plates_problem(19, 25, 1e-2, 1.3e-2, 2e4, seed=4, field_dependent=True,
                         source=W.SRC_TOWNSEND_ATTACH, n_species=3)
    _, _, st, n_ref, phi_ref, _, n_gpu, phi = run_both(avip, p, 25)
    for s in range(3):
        assert normwise(n_gpu[s], n_ref[s]) <= TOL, s
    assert normwise(phi, phi_ref) <= TOL


def test_pin_plane_small_parity(avip):
    """Needle anode geometry (the pin-plane shape at reduced size)."""
    p = W.plates_problem(41, 81, 1e-2, 2e-2, 2e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND,
                         needle_len=2e-3)
    _, _, st, n_ref, phi_ref, _, n_gpu, phi = run_both(avip, p, 20)
    for s in range(2):
        assert normwise(n_gpu[s], n_ref[s]) <= TOL
    assert normwise(phi, phi_ref) <= TOL


def test_graph_replay_equals_single_steps(avip):
    p = W.config_small(nx=25, ny=25, seed=12, source=W.SRC_TOWNSEND, voltage=2e4, field_dependent=True)
    a = avip.Mesh(p, rtol=1e-13)
    b = avip.Mesh(p, rtol=1e-13)
    a.run(12)
    for _ in range(12):
        b.step()
    np.testing.assert_array_equal(a.state(), b.state())


def test_checkpoint_resume_bitwise(avip):
    p = W.config_small(nx=21, ny=21, seed=13)
    a = avip.Mesh(p)
    a.run(5)
    snap = a.state()
    a.run(7)
    b = avip.Mesh(p)
    b.set_state(snap)
    b.run(7)
    np.testing.assert_array_equal(a.state(), b.state())


def test_checkpoint_rejects_bad_state_and_fills_given_buffer(avip):
    """state_set refuses a non-finite entry (AVIP_ENAN) or a history count outside 0..3
    (AVIP_EINVAL) and installs nothing; state_get fills a caller buffer (here pinned host memory)
    with the same values as a fresh array."""
    import torch
    p = W.config_small(nx=23, ny=19, seed=14)
    m = avip.Mesh(p)
    m.run(4)
    good = m.state()
    pinned = torch.empty(good.size, dtype=torch.float64, pin_memory=True).numpy()
    assert m.state(out=pinned) is pinned
    np.testing.assert_array_equal(pinned, good)
    with pytest.raises(ValueError):
        m.state(out=np.empty(good.size - 1))
    bad = good.copy()
    bad[7] = np.nan
    assert avip.state_set(m.h, bad) == avip.AVIP_ENAN
    bad = good.copy()
    bad[-1] = 4.0
    assert avip.state_set(m.h, bad) == avip.AVIP_EINVAL
    np.testing.assert_array_equal(m.state(), good)
    m.close()


def test_reorder_does_not_change_results(avip):
    p = W.config_small(nx=30, ny=22, seed=5)
    a = avip.Mesh(p, rtol=1e-14, reorder=1)
    b = avip.Mesh(p, rtol=1e-14, reorder=0)
    a.run(10)
    b.run(10)
    for s in range(2):
        assert normwise(a.density(s), b.density(s)) <= TOL


def test_torch_allocator_path(avip):
    import torch
    p = W.config_small(nx=17, ny=17, seed=21)
    before = torch.cuda.memory_allocated()
    m = avip.Mesh(p, use_torch_allocator=True)
    assert torch.cuda.memory_allocated() > before
    ref = avip.Mesh(p)
    m.run(3)
    ref.run(3)
    np.testing.assert_array_equal(m.state(), ref.state())
    m.close()
    assert torch.cuda.memory_allocated() == before


def test_error_paths(avip):
    p = W.config_small(nx=9, ny=9)
    o = avip.avip_opts_default()
    bad = p.tris.copy()
    bad[0, 0] = p.n_nodes + 5
    rc, _ = avip.mesh_create(p.xy, bad, p.node_bc, p.phi_D, o)
    assert rc == avip.AVIP_EINVAL
    deg = p.tris.copy()
    deg[0, 1] = deg[0, 0]
    rc, _ = avip.mesh_create(p.xy, deg, p.node_bc, p.phi_D, o)
    assert rc == avip.AVIP_EINVAL
    rc, _ = avip.mesh_create(p.xy, p.tris, np.zeros_like(p.node_bc), p.phi_D, o)
    assert rc == avip.AVIP_EINVAL
    rc, h = avip.mesh_create(p.xy, p.tris, p.node_bc, p.phi_D, o)
    assert rc == 0
    # stepping before any species is declared
    assert avip.dd_step(h, 0.0)[0] == avip.AVIP_ESTATE
    n0 = p.species[0].n0.copy()
    n0[3] = np.nan
    assert avip.species_set(h, 0, -1, 0, [0.04], 0.1, 0, n0) == avip.AVIP_ENAN
    assert avip.species_set(h, 1, -1, 0, [0.04], 0.1, 0, p.species[0].n0) == avip.AVIP_ESTATE
    assert avip.species_set(h, 0, 2, 0, [0.04], 0.1, 0, p.species[0].n0) == avip.AVIP_EINVAL
    assert avip.species_set(h, 0, -1, 0, [0.04], 0.1, 0, p.species[0].n0) == 0
    avip.mesh_destroy(h)
    # PCG iteration cap
    m = avip.Mesh(W.config_small(nx=33, ny=33), rtol=1e-15, max_iter=2)
    it, rr = m.poisson_solve(allow=(avip.AVIP_ENOTCONV,))
    assert it == 2 and rr > 1e-15


def test_tiny_and_single_slice_meshes(avip):
    """3 x 3 nodes (8 triangles, one partial slice) and 4 x 8 (exactly one 32-row slice)."""
    for nx, ny in ((3, 3), (4, 8)):
        p = W.config_small(nx=nx, ny=ny, seed=nx + ny, jitter=0.0)
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(3)
        m = avip.Mesh(p, rtol=1e-14)
        m.run(3)
        for s in range(2):
            assert normwise(m.density(s), n_ref[s]) <= TOL
        assert normwise(m.phi(), phi_ref) <= TOL


# ---------------------------------------------------------------- mixed precision
MIXED_TOL = 1e-6


@pytest.mark.parametrize("kind", [0, 6, 1])
def test_mixed_poisson_matches_oracle(avip, kind):
    """FP32 inner solve + FP64 refinement reaches the FP64 answer (rtol 1e-12 on the
    residual): the one-cluster AMG form (kind 0 picks it for this size), the one-cluster Jacobi
    form (6) and the grid-wide Jacobi kernel (1, reported as 4)."""
    p = W.config_small(nx=40, ny=33, seed=5)
    o = O.Oracle(p)
    phi_ref = o.poisson(o.initial_state())
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-12, pcg_kind=kind)
    assert m.info["pcg_kind"] == {0: 11, 6: 6, 1: 4}[kind]
    it, rr = m.poisson_solve()
    assert rr <= 1e-12
    assert normwise(m.phi(), phi_ref) <= 1e-10


@pytest.mark.parametrize("scheme,nsteps", [(W.FLUX_SG, 2000), (W.FLUX_LLW, 1000)])
def test_mixed_plates65_within_1e6(avip, scheme, nsteps):
    """Mixed precision on the 65 x 65 plates mesh and physics (FP32 gradients, fluxes and inner
    PCG, FP64 refinement of the Poisson residual to 1e-10): phi, n_e and n_+ within 1e-6
    (norm-wise) of the FP64 oracle.  2000 steps with the Scharfetter-Gummel flux; 1000 with
    limited Lax-Wendroff, whose unclipped FP64 solution of this case develops negative electron
    densities at the trailing edge from step ~600 that the dielectric relaxation amplifies
    until the run blows up near step 1600 (the oracle does the same), so that later steps
    amplify any rounding difference."""
    p = W.config_plates_65()
    p.opts.scheme = scheme
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    errs = [normwise(m.density(s), n_ref[s]) for s in range(2)] + [normwise(m.phi(), phi_ref)]
    print("mixed-precision %d-step norm-wise errors (n_e, n_+, phi), scheme %d:" % (nsteps, scheme), errs)
    assert max(errs) <= MIXED_TOL


@pytest.mark.parametrize("scheme,nsteps", [(W.FLUX_LLW, 300), (W.FLUX_SG, 200)])
def test_mixed_fp32_drift_diffusion_within_1e6(avip, scheme, nsteps):
    """Mixed precision also runs gradients, velocities, sources and fluxes in FP32 (FP64 state,
    update, time step and charge): field-dependent mobility, Townsend ionisation, outflow
    closure, both flux schemes, within 1e-6 of the FP64 oracle.  The Scharfetter-Gummel run
    stops at 200 steps: its centred normal part is anti-diffusive for the ions (cell Peclet
    ~2e4), and a CPU run of the oracle with only the SG fluxes rounded to FP32 departs from the
    FP64 oracle by 1.3e-8 at step 200 but 1.8e-6 at step 300 (an FP32 property of the scheme on
    this case, not of the kernel)."""
    p = W.plates_problem(41, 37, 1e-2, 0.9e-2, 2.5e4, seed=23, field_dependent=True, source=W.SRC_TOWNSEND)
    p.opts.scheme = scheme
    p.species[0].bnd_mode = W.BND_OUTFLOW
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    errs = [normwise(m.density(s), n_ref[s]) for s in range(2)] + [normwise(m.phi(), phi_ref)]
    print("mixed FP32-DD %d-step norm-wise errors (n_e, n_+, phi), scheme %d:" % (nsteps, scheme), errs)
    assert max(errs) <= MIXED_TOL
    assert abs(st["t"] - sum(dts)) <= 1e-6 * sum(dts)


def test_mixed_three_species_within_1e6(avip):
    p = W.plates_problem(29, 31, 1e-2, 1e-2, 2e4, seed=24, field_dependent=True,
                         source=W.SRC_TOWNSEND_ATTACH, n_species=3)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(100)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10)
    assert m.run(100)["status"] == 0
    for s in range(3):
        assert normwise(m.density(s), n_ref[s]) <= MIXED_TOL, s


@pytest.mark.parametrize("kind", [1, 2, 5])
def test_every_pcg_kernel_matches_oracle(avip, kind):
    """Streaming (1), register-resident (2) and cluster-resident (5) FP64 solvers, forced on a
    mesh of 71 x 53 nodes (ragged last slice), give the oracle's step."""
    p = W.plates_problem(71, 53, 1e-2, 0.8e-2, 1.5e4, seed=31, field_dependent=True, source=W.SRC_TOWNSEND)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(6)
    m = avip.Mesh(p, rtol=1e-13, pcg_kind=kind)
    m.run(6)
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL
    assert normwise(m.phi(), phi_ref) <= TOL


def test_neumann_marker_same_as_free(avip):
    """node_bc = 2 on the side nodes gives bit-identical results to 0 (the natural condition)."""
    import dataclasses
    p = W.config_small(nx=21, ny=19, seed=4)
    bc2 = p.node_bc.copy()
    ii = np.tile(np.arange(21), 19)
    bc2[((ii == 0) | (ii == 20)) & (p.node_bc == 0)] = 2
    a = avip.Mesh(p)
    b = avip.Mesh(dataclasses.replace(p, node_bc=bc2))
    a.run(5)
    b.run(5)
    np.testing.assert_array_equal(a.state(), b.state())
    a.close()
    b.close()


def test_fp64_closure_math_matches_cuda_math_library(avip):
    """The library's own FP64 exp / log / pow (the local-field mobility and Townsend closures)
    and reciprocal (the limiter ratio) against the CUDA math library and the IEEE quotient: exp
    and log within a few ulp; pow within 4e-16 (1 + |p ln x|) with |p ln x| <= 2.3 ln(1.3e6)
    here, i.e. about 1.5e-14; the reciprocal within two ulp."""
    rc, err = avip.fp64_math_check()
    assert rc == avip.AVIP_OK
    assert err[0] <= 1.2e-15, err
    assert err[1] <= 1.2e-15, err
    assert err[2] <= 4e-16 * (1.0 + 2.3 * np.log(1.3e6)), err
    assert err[3] <= 4.5e-16, err  # two Newton steps: within two ulp of the quotient
