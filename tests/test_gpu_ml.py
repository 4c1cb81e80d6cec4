"""Parity of the GPU path with the FP64 oracle for the three-species air chemistry (ionisation,
field-dependent attachment, electron-ion and ion-ion recombination, immobile ions) and the
linear electrode-voltage ramp: the ramped potential of a charge-free gap on every planar
solver, steps through the ramp on triangle and hybrid meshes with LLW and SG, mixed precision,
and a batch whose instances sit at different times of their ramps.  Tolerances: 1e-12 on a
lone solve, 1e-10 after steps (FP64), 1e-6 for mixed precision."""
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


def ml(nx=41, ny=41, **kw):
    kw.setdefault("needle_len", 1e-3)
    return W.morrow_lowke_problem(nx, ny, 5e-3, 5e-3, 5e3, seed=7, **kw)


@pytest.mark.parametrize("kind", [1, 2, 5, 8, 11])
def test_ramped_potential_of_a_charge_free_gap(avip, kind):
    """dt fixed at v_rise / 8: after k steps phi = min(k / 8, 1) V y / L (no needle)."""
    p = ml(33, 29, needle_len=0.0, n_back=0.0)
    p.opts.dt_fixed = 2e-9 / 8
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=kind)
    assert m.info["pcg_kind"] == kind
    for k in range(10):
        m.poisson_solve()
        g = min(k / 8.0, 1.0)
        ref = g * 5e3 * p.xy[:, 1] / 5e-3
        if g == 0.0:
            assert np.abs(m.phi()).max() == 0.0
        else:
            assert normwise(m.phi(), ref) <= 1e-12, (k, kind)
        m.step()
    m.close()


@pytest.mark.parametrize("scheme,frac", [(W.FLUX_LLW, 0.0), (W.FLUX_SG, 0.0), (W.FLUX_LLW, 0.5), (W.FLUX_SG, 1.0)])
def test_ml_steps_through_the_ramp(avip, scheme, frac):
    """40 automatic steps from a Gaussian seed below the needle while the anode rises (the
    first steps at a few volts, the chemistry switching on as the field grows)."""
    p = ml(quad_fraction=frac, v_rise=2e-10)
    p.species[0].n0[:] = W.gaussian(p.xy, 2.5e-3, 3.5e-3, 3e-4, 1e19, 1e15)
    p.species[1].n0[:] = p.species[0].n0
    p.opts.scheme = scheme
    nsteps = 40
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, rtol=1e-13)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(3):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n_ref)
    assert abs(st["charge"] - o.charge(n_ref)) <= 1e-10 * scale
    m.close()


def test_ml_large_mesh_amg(avip):
    """A 40,401-node mesh on the automatic AMG solver, 10 steps into the ramp."""
    p = ml(201, 201, v_rise=1e-10)
    p.species[0].n0[:] = W.gaussian(p.xy, 2.5e-3, 3.5e-3, 3e-4, 1e19, 1e15)
    p.species[1].n0[:] = p.species[0].n0
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


def test_ml_mixed_within_1e6(avip):
    p = ml(v_rise=2e-10)
    p.species[0].n0[:] = W.gaussian(p.xy, 2.5e-3, 3.5e-3, 3e-4, 1e19, 1e15)
    p.species[1].n0[:] = p.species[0].n0
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(40)
    m = avip.Mesh(p, precision=avip.PREC_MIXED, rtol=1e-10)
    st = m.run(40)
    assert st["status"] == 0
    errs = [normwise(m.density(s), n_ref[s]) for s in range(3)] + [normwise(m.phi(), phi_ref)]
    assert max(errs) <= 1e-6, errs
    m.close()


def test_ml_batch_instances_keep_their_own_time(avip):
    """Two ramped instances, one advanced 5 steps alone first: in the batch each solve uses its
    own simulated time (the per-instance device scalars), so both equal their oracle runs."""
    ps = [ml(29, 27, v_rise=1e-10), ml(33, 25, v_rise=3e-10), W.config_small(nx=21, ny=19, seed=4)]
    for p in ps[:2]:
        p.species[0].n0[:] = W.gaussian(p.xy, 2.5e-3, 3.5e-3, 3e-4, 1e19, 1e15)
        p.species[1].n0[:] = p.species[0].n0
    meshes = [avip.Mesh(p, rtol=1e-13, pcg_kind=5) for p in ps]
    meshes[0].run(5)
    b = avip.Batch(meshes)
    b.run(6)
    for k, p in enumerate(ps):
        o = O.Oracle(p)
        n_ref, phi_ref, _ = o.run(11 if k == 0 else 6)
        for s in range(len(p.species)):
            assert normwise(meshes[k].density(s), n_ref[s]) <= TOL, (k, s)
        assert normwise(meshes[k].phi(), phi_ref) <= TOL, k
    b.close()
