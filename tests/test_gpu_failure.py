"""Failure detection on the GPU without faulting it: a grid-barrier wait that runs out (the
handle's wait_timeout set to 0, so the first block that has to wait gives up at once) and the
device-side check of non-finite densities (a time step so large that the explicit update
overflows to infinity).  Both end in a status code; the handle then steps correctly again."""
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


def test_wait_timeout_expires_then_handle_recovers(avip):
    # 201 x 201 nodes: the cooperative AMG-preconditioned CG over the whole GPU (kind 8)
    p = W.plates_problem(201, 201, 1e-2, 1e-2, 2e4, seed=31, field_dependent=True, source=W.SRC_TOWNSEND)
    m = avip.Mesh(p, rtol=1e-13, wait_timeout=0.0)
    assert m.info["pcg_kind"] == 8 and m.info["pcg_blocks"] > 1
    s0 = m.state()
    st = m.run(1, allow=(avip.AVIP_ETIMEOUT,))
    assert st["status"] == avip.AVIP_ETIMEOUT
    rc, _, _ = avip.poisson_solve(m.h)
    assert rc == avip.AVIP_ETIMEOUT
    # a normal limit again: the same handle, from the saved state, matches the oracle
    m.set_wait_timeout(2.0)
    m.set_state(s0)
    st = m.run(3)
    assert st["status"] == avip.AVIP_OK and st["steps"] == 3
    n_ref, phi_ref, _ = O.Oracle(p).run(3)
    assert normwise(m.phi(), phi_ref) <= 1e-10
    for s in range(2):
        assert normwise(m.density(s), n_ref[s]) <= 1e-10
    with pytest.raises(avip.AvipError):
        m.set_wait_timeout(-1.0)
    m.close()


def test_device_nan_check_then_handle_recovers(avip):
    p = W.config_small(nx=21, ny=19, seed=5, voltage=1e4)
    m = avip.Mesh(p, rtol=1e-13)
    s0 = m.state()
    # finite on the host, infinite after the update: only the device check can see it
    rc, used = avip.dd_step(m.h, 1e300)
    assert rc == avip.AVIP_ENAN and used == 1e300
    d = m.density(0)
    assert not np.all(np.isfinite(d))
    m.set_state(s0)
    st = m.run(2)
    assert st["status"] == avip.AVIP_OK
    n_ref, phi_ref, _ = O.Oracle(p).run(2)
    assert normwise(m.density(0), n_ref[0]) <= 1e-10
    assert normwise(m.phi(), phi_ref) <= 1e-10
    m.close()
