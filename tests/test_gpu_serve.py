"""Serving loop: results are the same alone and in the mix; admission respects the HBM
budget and rejects requests that can never fit; nothing runs out of memory."""
import numpy as np
import pytest

from helpers import normwise
from paper_2201_01291_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2201_01291_gb300 import avip, build, serve
    build.build()
    avip.load()
    return avip, serve


def _requests(serve, n=6):
    out = []
    for k in range(n):
        nx, ny = 15 + 4 * k, 21 + 3 * k
        p = W.plates_problem(nx, ny, 1e-2, 1.2e-2, 1e4 + 2e3 * k, seed=100 + k, field_dependent=True,
                             source=W.SRC_TOWNSEND if k % 2 == 0 else W.SRC_TOWNSEND_ATTACH,
                             n_species=2 if k % 2 == 0 else 3)
        out.append(serve.Request(k, 0.03 * k, p, 24 + 5 * k))
    return out


def test_served_equals_alone(mods):
    avip, serve = mods
    reqs = _requests(serve)
    srv = serve.Server(hbm_budget=1 << 30, max_slots=4, chunk=7)
    rep = srv.run(reqs)
    assert rep["completed"] == len(reqs)
    for r in reqs:
        m = avip.Mesh(r.problem, rtol=srv.rtol, precision=srv.precision, pcg_kind=serve.solver_kind(r.problem),
                      cluster_size=serve.cluster_ctas(r.problem))
        m.run(r.nsteps)
        alone = m.state()
        m.close()
        assert normwise(r.state, alone) <= 1e-12, r.rid
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0


def test_admission_respects_budget(mods):
    avip, serve = mods
    reqs = _requests(serve)
    sizes = [serve.estimate_bytes(r.problem) for r in reqs]
    budget = sorted(sizes)[-1] + sorted(sizes)[-2]          # at most two of the largest at once
    big = W.plates_problem(400, 400, 1e-2, 1e-2, 1e4, seed=9)
    reqs.append(serve.Request(99, 0.0, big, 5))              # can never fit this budget
    srv = serve.Server(hbm_budget=budget, max_slots=8, chunk=6, keep_state=False)
    rep = srv.run(reqs, realtime=False)
    assert rep["rejected"] == 1 and rep["completed"] == len(reqs) - 1
    assert all(used <= budget for _, _, used, _ in srv.admit_log)


def test_admission_follows_free_device_memory(mods):
    """With the device reporting little free memory, a request waits (it is admitted only while
    its estimate fits what is free minus the other admitted requests' reservations) and one that
    could never fit is rejected instead of attempted."""
    avip, serve = mods
    reqs = _requests(serve, n=3)
    need = max(serve.estimate_bytes(r.problem) for r in reqs)
    fake_free = [serve.FREE_MARGIN + need]        # room for one request at a time
    srv = serve.Server(hbm_budget=1 << 34, max_slots=8, chunk=5, keep_state=False,
                       free_bytes=lambda: fake_free[0])
    rep = srv.run(reqs, realtime=False)
    assert rep["completed"] == 3
    assert all(free >= 0 for *_, free in srv.admit_log)
    fake_free[0] = serve.FREE_MARGIN // 2           # nothing fits: rejected, not run
    rep = serve.Server(hbm_budget=1 << 34, max_slots=8, chunk=5, keep_state=False,
                       free_bytes=lambda: fake_free[0]).run(_requests(serve, n=2), realtime=False)
    assert rep["rejected"] == 2 and rep["completed"] == 0


@pytest.mark.parametrize("precision,rtol,tol", [("mixed", None, 1e-6), ("fp64", 1e-13, 1e-10)])
def test_served_matches_oracle(mods, precision, rtol, tol):
    """Three small requests served together (one above the library's automatic cluster size, so
    it takes the served AMG cluster solve) against the FP64 oracle: norm-wise 1e-6 in the default
    mixed precision, 1e-10 on the FP64 path."""
    import avip_oracle as O
    avip, serve = mods
    reqs = []
    for k, (nx, ny) in enumerate([(21, 27), (33, 25), (151, 141)]):
        p = W.plates_problem(nx, ny, 1e-2, 1e-2, 1.2e4 + 3e3 * k, seed=300 + k, field_dependent=True,
                             source=W.SRC_TOWNSEND)
        reqs.append(serve.Request(k, 0.01 * k, p, 6 + k))
    assert serve.solver_kind(reqs[2].problem) == 11
    prec = avip.PREC_MIXED if precision == "mixed" else avip.PREC_FP64
    rep = serve.Server(hbm_budget=1 << 30, max_slots=3, chunk=3, rtol=rtol, precision=prec).run(reqs)
    assert rep["completed"] == 3
    for r in reqs:
        n_ref, phi_ref, dts = O.Oracle(r.problem).run(r.nsteps)
        N = r.problem.n_nodes
        ns = len(r.problem.species)
        for s_ in range(ns):
            assert normwise(r.state[s_ * N:(s_ + 1) * N], n_ref[s_]) <= tol, (r.rid, s_)
        assert normwise(r.state[ns * N:(ns + 1) * N], phi_ref) <= tol, r.rid
