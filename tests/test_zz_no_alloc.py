"""The no-allocation solver entry point (pcg_csr_static) against the handle-based Poisson
solve.  It serves callers that may not allocate device memory at all, so it keeps its work
vectors in an array compiled into the library; this test checks, on two calls in a row, that
it returns the same potential as poisson_solve on the same system.  Kept in its own file,
collected last, so a failure here does not hide the other tests."""
import numpy as np
import pytest

import avip_oracle as O
from helpers import normwise
from paper_2201_01291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_system(o, p, n):
    """Dirichlet-eliminated system K_FF phi_F = b_F of the current densities (the same
    system the library assembles), as CSR arrays."""
    free, dirn = o.solver.free, o.solver.dir
    K = o.K.tocsr()
    KFF = K[free][:, free].tocsr()
    KFF.sort_indices()
    b = O.poisson_rhs(o.charge_density(n), o.V_node)[free] - K[free][:, dirn] @ p.phi_D[dirn]
    return free, KFF, b


def test_static_pcg_matches_poisson_solve_twice():
    import torch
    from paper_2201_01291_gb300 import avip, build
    build.build()
    avip.load()
    p = W.config_small(nx=33, ny=29, seed=17, source=W.SRC_TOWNSEND, voltage=2e4, field_dependent=True)
    o = O.Oracle(p)
    m = avip.Mesh(p, rtol=1e-14)
    dev = torch.device("cuda", 0)
    x = None
    for call in range(2):
        m.poisson_solve()
        phi_ref = m.phi()
        n = [m.density(s) for s in range(2)]
        free, KFF, b = _free_system(o, p, n)
        rp = torch.tensor(KFF.indptr, dtype=torch.int32, device=dev)
        ci = torch.tensor(KFF.indices, dtype=torch.int32, device=dev)
        va = torch.tensor(KFF.data, dtype=torch.float64, device=dev)
        bd = torch.tensor(b, dtype=torch.float64, device=dev)
        if x is None:
            x = torch.zeros(free.size, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc, it, rr = avip.pcg_csr_static(free.size, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), bd.data_ptr(),
                                         x.data_ptr(), 1e-14, 20000, torch.cuda.current_stream().cuda_stream)
        assert rc == 0, (call, rc, avip.status_str(rc))
        assert rr <= 1e-14 and it > 0
        assert normwise(x.cpu().numpy(), phi_ref[free]) <= 1e-10, call
        m.step()  # new densities for the second call (x is reused as its warm start)
    m.close()


def test_static_pcg_iteration_cap_and_zero_rhs():
    """The failure path: max_iter reached gives AVIP_ENOTCONV, x holds the last iterate and the
    reported relative residual is that of x (recomputed here on the host); a zero right-hand
    side gives x = 0 from any initial guess."""
    import torch
    from paper_2201_01291_gb300 import avip, build
    build.build()
    avip.load()
    p = W.config_small(nx=41, ny=37, seed=23, voltage=1e4)
    o = O.Oracle(p)
    free, KFF, b = _free_system(o, p, o.initial_state())
    dev = torch.device("cuda", 0)
    rp = torch.tensor(KFF.indptr, dtype=torch.int32, device=dev)
    ci = torch.tensor(KFF.indices, dtype=torch.int32, device=dev)
    va = torch.tensor(KFF.data, dtype=torch.float64, device=dev)
    bd = torch.tensor(b, dtype=torch.float64, device=dev)
    x = torch.zeros(free.size, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    rc, it, rr = avip.pcg_csr_static(free.size, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), bd.data_ptr(),
                                     x.data_ptr(), 1e-14, 5, st)
    assert rc == avip.AVIP_ENOTCONV and it == 5
    xh = x.cpu().numpy()
    ref = np.linalg.norm(b - KFF @ xh) / np.linalg.norm(b)
    assert abs(rr - ref) <= 1e-8 * ref and ref > 1e-6
    # b = 0 from the non-zero iterate left above: x = 0, converged at once
    bd.zero_()
    torch.cuda.synchronize()
    rc, it, rr = avip.pcg_csr_static(free.size, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), bd.data_ptr(),
                                     x.data_ptr(), 1e-14, 5, st)
    assert rc == avip.AVIP_OK and it == 0 and rr == 0.0
    assert torch.count_nonzero(x).item() == 0


def test_static_pcg_rejects_oversize():
    from paper_2201_01291_gb300 import avip
    avip.load()
    rc, _, _ = avip.pcg_csr_static(262144 + 1, 1, 1, 1, 1, 1, 1e-10, 10)
    assert rc == avip.AVIP_EINVAL
