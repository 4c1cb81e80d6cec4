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
        m = avip.Mesh(r.problem, rtol=1e-12)
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
    assert all(used <= budget for _, _, used in srv.admit_log)
