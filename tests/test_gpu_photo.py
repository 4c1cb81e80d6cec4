"""Parity of the photoionisation source on the GPU (three Helmholtz solves per step by the
handle's own solver kind) with the FP64 oracle: the source S_ph of one step with every FP64
solver kind (planar and axisymmetric), steps with photoionisation on both geometries, a large
axisymmetric mesh on the AMG-preconditioned BiCGStab, and the error paths.  Tolerances: 1e-10
norm-wise on S_ph, phi and the densities (solves at rtol 1e-14: the Helmholtz terms with small
kappa are as ill-conditioned as the Poisson problem), except S_ph on the large mesh (below)."""
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


def planar(nx=33, ny=31, **kw):
    p = W.plates_problem(nx, ny, 1e-2, 1e-2, 2.5e4, seed=9, field_dependent=True, source=W.SRC_TOWNSEND,
                         n_back=1e9, **kw)
    return W.dataclasses.replace(p, photo=W.photo_air())


def axisym(nx=33, nr=29, **kw):
    p = W.axisym_problem(nx, nr, 1.25e-2, 1.25e-2, 18750.0, seed=5, n_peak=5e18, n_back=1e9, sigma=4e-4,
                         field_dependent=True, source=W.SRC_TOWNSEND, x0=1e-2, **kw)
    return W.dataclasses.replace(p, photo=W.photo_air())


@pytest.mark.parametrize("geom,kind", [("planar", 1), ("planar", 2), ("planar", 5), ("planar", 8),
                                       ("planar", 11), ("axisym", 7), ("axisym", 9)])
def test_photo_source_one_step(avip, geom, kind):
    p = planar() if geom == "planar" else axisym()
    o = O.Oracle(p)
    n1, info = o.step(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14, pcg_kind=kind)
    assert m.info["pcg_kind"] == kind
    dt = m.step()
    # the chemical limit divides by S_ph, an iterative solve's output: the solve bar applies
    assert abs(dt - info["dt"]) <= TOL * info["dt"]
    assert o.last_photo.max() > 0
    assert normwise(m.photo(), o.last_photo) <= TOL
    for s in range(2):
        assert normwise(m.density(s), n1[s]) <= TOL, s
    ps = m.photo_stats()
    # the whole-GPU AMG kinds solve the three terms side by side, each on its own blocks
    assert ps["side_by_side"] == (kind in (8, 9) and m.info["pcg_blocks"] >= 3)
    assert len(ps["iters"]) == 3 and all(k > 0 for k in ps["iters"])
    assert all(r <= 1e-14 for r in ps["relres"]), ps
    m.close()


@pytest.mark.parametrize("geom", ["planar", "axisym"])
def test_photo_steps_parity(avip, geom):
    p = planar(41, 39) if geom == "planar" else axisym(41, 33)
    nsteps = 20
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, rtol=1e-14)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= TOL * sum(dts)
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    assert normwise(m.photo(), o.last_photo) <= TOL
    m.close()


def test_photo_large_axisymmetric_amg(avip):
    """40,000 nodes: the automatic AMG-preconditioned BiCGStab for the Poisson and the three
    Helmholtz problems (each with its own hierarchy), 6 steps."""
    p = axisym(201, 201)
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(6)
    m = avip.Mesh(p, rtol=1e-13)
    assert m.info["pcg_kind"] == 9
    st = m.run(6)
    assert st["status"] == 0
    ps = m.photo_stats()
    assert ps["side_by_side"] and all(r <= 1e-13 for r in ps["relres"]), ps
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    # S_ph is the output of a solve stopped at rtol 1e-13 (BiCGStab stagnates before 1e-14 on
    # this mesh): its accuracy is the solve's, 3e-10 measured, and it enters the densities
    # only through dt S_ph
    assert normwise(m.photo(), o.last_photo) <= 1e-9
    m.close()


def test_photo_error_paths(avip):
    p = planar(21, 19)
    ph = p.photo
    q = W.dataclasses.replace(p, photo=None)
    mixed = avip.Mesh(q, precision=avip.PREC_MIXED)
    assert avip.photo_set(mixed.h, ph.a, ph.kappa, ph.c) == avip.AVIP_EINVAL
    mixed.close()
    m = avip.Mesh(q)
    assert avip.photo_set(m.h, ph.a, [-1.0, 2.0, 3.0], ph.c) == avip.AVIP_EINVAL
    assert avip.photo_set(m.h, ph.a, ph.kappa, ph.c) == avip.AVIP_OK
    assert avip.photo_set(m.h, ph.a, ph.kappa, ph.c) == avip.AVIP_ESTATE
    with pytest.raises(avip.AvipError):
        avip.Batch([m])
    m.close()
    plain = avip.Mesh(q)  # no photoionisation: no terms, nothing side by side
    assert plain.photo_stats() == {"iters": [], "relres": [], "side_by_side": False}
    plain.close()


def test_photo_on_hybrid_mesh_with_chemistry_and_ramp(avip):
    """Photoionisation with the three-species chemistry and the voltage ramp on a hybrid
    triangle/quadrangle mesh (the second case of smoke())."""
    q = W.morrow_lowke_problem(23, 21, 5e-3, 5e-3, 5e3, seed=3, needle_len=1e-3, quad_fraction=0.5, v_rise=2e-10)
    q.species[0].n0[:] = W.gaussian(q.xy, 2.5e-3, 3.5e-3, 3e-4, 1e19, 1e15)
    q.species[1].n0[:] = q.species[0].n0
    q = W.dataclasses.replace(q, photo=W.photo_air(p_torr=760.0 * 300.0 / 1000.0))
    o = O.Oracle(q)
    n_ref, phi_ref, _ = o.run(12)
    m = avip.Mesh(q, rtol=1e-14)
    st = m.run(12)
    assert st["status"] == 0
    for s in range(3):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.photo(), o.last_photo) <= TOL
    m.close()


def test_photo_side_by_side_skips_after_timeout_then_recovers(avip):
    """With a wait limit of zero the Poisson solve gives up; the side-by-side photoionisation
    launch that follows sees the failed run and every group leaves together (none waits for a
    group that skipped).  With a normal limit the same handle matches the oracle."""
    p = planar(121, 117)
    m = avip.Mesh(p, rtol=1e-13, pcg_kind=8, wait_timeout=0.0)
    assert m.photo_stats()["side_by_side"]
    s0 = m.state()
    st = m.run(1, allow=(avip.AVIP_ETIMEOUT,))
    assert st["status"] == avip.AVIP_ETIMEOUT
    m.set_wait_timeout(2.0)
    m.set_state(s0)
    st = m.run(2)
    assert st["status"] == avip.AVIP_OK
    o = O.Oracle(p)
    n_ref, phi_ref, _ = o.run(2)
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    # S_ph is the output of solves stopped at rtol 1e-13: the solve's accuracy
    assert normwise(m.photo(), o.last_photo) <= 1e-9
    m.close()


def test_photo_side_by_side_on_the_whole_grid(avip):
    """A planar mesh large enough for the whole-GPU AMG grid (one block per SM): the three terms
    run side by side on groups of about a third of the SMs each, every term converges to the
    handle's tolerance and the run status stays OK (no group waits on another)."""
    p = planar(421, 421)
    m = avip.Mesh(p, rtol=1e-12)
    assert m.info["pcg_kind"] == 8
    st = m.run(2)
    assert st["status"] == avip.AVIP_OK and st["steps"] == 2
    ps = m.photo_stats()
    assert ps["side_by_side"] and m.info["pcg_blocks"] >= 100, (ps, m.info)
    assert all(k > 0 for k in ps["iters"]) and all(r <= 1e-12 for r in ps["relres"]), ps
    assert np.all(np.isfinite(m.photo())) and m.photo().max() > 0
    m.close()
