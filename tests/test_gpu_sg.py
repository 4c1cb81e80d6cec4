"""Parity of the Scharfetter-Gummel edge flux on the GPU (opts.scheme = AVIP_FLUX_SG) with the
FP64 oracle: planar and axisymmetric meshes, field-dependent mobility, Townsend ionisation,
both boundary closures; and a batch of SG instances equal to the same instances alone.
Tolerance: norm-wise 1e-10 on phi and every density."""
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


def sg(p):
    p.opts.scheme = W.FLUX_SG
    return p


def check(avip, p, nsteps, rtol=1e-13):
    o = O.Oracle(p)
    n_ref, phi_ref, dts = o.run(nsteps)
    m = avip.Mesh(p, rtol=rtol)
    st = m.run(nsteps)
    assert st["steps"] == nsteps and st["status"] == 0
    assert abs(st["t"] - sum(dts)) <= 1e-12 * sum(dts)
    for s in range(len(p.species)):
        assert normwise(m.density(s), n_ref[s]) <= TOL, s
    assert normwise(m.phi(), phi_ref) <= TOL
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n_ref)
    assert abs(st["charge"] - o.charge(n_ref)) <= 1e-10 * scale
    m.close()


def test_sg_single_step(avip):
    p = sg(W.config_small(nx=21, ny=19, seed=3))
    o = O.Oracle(p)
    n1, info = o.step(o.initial_state())
    m = avip.Mesh(p, rtol=1e-14)
    dt = m.step()
    assert abs(dt - info["dt"]) <= 1e-12 * info["dt"]
    for s in range(2):
        assert normwise(m.density(s), n1[s]) <= TOL
    m.close()


@pytest.mark.parametrize("bnd", [W.BND_NEUMANN, W.BND_OUTFLOW])
def test_sg_plates_townsend_parity(avip, bnd):
    p = sg(W.plates_problem(33, 29, 1e-2, 0.9e-2, 2.5e4, seed=12, field_dependent=True, source=W.SRC_TOWNSEND))
    p.species[0].bnd_mode = bnd
    check(avip, p, 50)


def test_sg_plates65_100_steps(avip):
    check(avip, sg(W.config_plates_65()), 100)


def test_sg_axisym_parity(avip):
    p = sg(W.axisym_problem(37, 25, 1e-2, 0.6e-2, 2.5e4, seed=13, field_dependent=True, source=W.SRC_TOWNSEND))
    check(avip, p, 40)


def test_sg_three_species_parity(avip):
    p = sg(W.plates_problem(27, 23, 1e-2, 1e-2, 2e4, seed=14, field_dependent=True,
                            source=W.SRC_TOWNSEND_ATTACH, n_species=3))
    check(avip, p, 25)


def test_sg_batch_equals_alone(avip):
    probs = [sg(W.plates_problem(n, n + 4, 1e-2, 1e-2, 1.5e4 + 1e3 * n, seed=40 + n, field_dependent=True,
                                 source=W.SRC_TOWNSEND)) for n in (11, 19, 27)]
    alone = []
    for p in probs:
        m = avip.Mesh(p, rtol=1e-12, pcg_kind=5)
        m.run(15)
        alone.append([m.density(s) for s in range(2)])
        m.close()
    ms = [avip.Mesh(p, rtol=1e-12, pcg_kind=5) for p in probs]
    b = avip.Batch(ms, cluster_size=16)
    b.run(15)
    for k, m in enumerate(ms):
        for s in range(2):
            assert normwise(m.density(s), alone[k][s]) <= 1e-12
    b.close()
    for m in ms:
        m.close()
