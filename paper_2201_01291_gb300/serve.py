"""Serving loop for discharge solves (continuous batching on one GPU).

Requests (a discharge problem and a number of explicit steps) arrive over time.  The server
admits a request as soon as it has arrived, a slot is free and its device memory fits: the
request's estimate must fit both the server's HBM budget and the device memory free at that
moment (cudaMemGetInfo) minus the reservations of admitted requests whose handle is not built
yet.  The request then keeps its whole state resident on the device (one mesh handle with its
own CUDA stream) until its last step, and releases slot and memory when done, which admits the
requests waiting behind it.  Admitted requests advance in chunks of steps on worker threads;
the CUDA work of concurrent requests overlaps on the device: every request of up to
SHARED_MAX_NODES nodes solves its Poisson problem on one thread-block cluster (the Jacobi or
AMG-preconditioned cluster solvers, 16 CTAs for the AMG ones), so up to nine of them run side by
side on the 152 SMs.
Larger requests use the whole-GPU cooperative kernel and run their chunks exclusively, because
a cooperative launch must have its whole grid resident.

Requests run in mixed precision by default (FP32 inner CG and V-cycle with FP64 refinement of
the Poisson residual, FP32 drift-diffusion fluxes, FP64 state, time step and charge): the
served form of the task is held to 1e-6 of the FP64 oracle, like the mixed-precision and
batched forms; `precision=avip.PREC_FP64` serves the plain FP64 path.  The numerics are the
library's: a request gives the same result alone and in the mix.
Latency of a request = completion time - arrival time; the report gives p50/p99 latency and
the aggregate cell-steps/s (triangles x steps of all requests / makespan).
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import List, Optional

import numpy as np

from . import avip

# Device bytes of one handle, per node and per stored matrix entry (SELL elements plus the
# per-node vectors of the solver and of the drift-diffusion stage); used for admission.
BYTES_PER_NODE = 1400
BYTES_PER_TRI = 24
SHARED_MAX_NODES = 300000  # requests up to this size solve on one thread-block cluster (shared)
AUTO_CLUSTER_NODES = 20000  # below this the library's automatic choice is already a cluster solver
CLUSTER_KINDS = (5, 6, 11)  # solver kinds that occupy one thread-block cluster, not the whole GPU
FREE_MARGIN = 512 << 20  # device memory kept free for the CUDA runtime and the caching allocator
# CTAs of a served request's cluster, by size.  On the 100-request sample of the served
# benchmark, 16 CTAs for every shared request gave 2.40e8 cell-steps/s; 4 CTAs for all 9.3e7,
# 4 / 8 / 16 by size 1.80e8 (small clusters make the large requests the tail of the makespan).
CLUSTER_CTAS_BY_NODES = ((SHARED_MAX_NODES, 16),)


def estimate_bytes(problem) -> int:
    return int(problem.n_nodes * BYTES_PER_NODE + problem.n_tris * BYTES_PER_TRI) + (1 << 20)


def solver_kind(problem) -> int:
    """pcg_kind for a served request: the AMG solve on one cluster (11) for the mid-size meshes
    the library would give the whole GPU, the library's choice (0) otherwise."""
    return 11 if AUTO_CLUSTER_NODES < problem.n_nodes <= SHARED_MAX_NODES else 0


def cluster_ctas(problem) -> int:
    """CTAs of the cluster a served request solves on (see CLUSTER_CTAS_BY_NODES); 0 = the
    library's choice."""
    for max_nodes, ctas in CLUSTER_CTAS_BY_NODES:
        if problem.n_nodes <= max_nodes:
            return ctas
    return 0


def device_free_bytes() -> int:
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    problem: object
    nsteps: int
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    state: Optional[np.ndarray] = None
    status: int = 0
    pcg_iters: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _GpuLock:
    """Shared (cluster-sized requests) / exclusive (whole-GPU requests) lock."""

    def __init__(self):
        self.cv = threading.Condition()
        self.shared = 0
        self.exclusive = False
        self.waiting_exclusive = 0

    def acquire(self, exclusive: bool):
        with self.cv:
            if exclusive:
                self.waiting_exclusive += 1
                self.cv.wait_for(lambda: not self.exclusive and self.shared == 0)
                self.waiting_exclusive -= 1
                self.exclusive = True
            else:
                self.cv.wait_for(lambda: not self.exclusive and self.waiting_exclusive == 0)
                self.shared += 1

    def release(self, exclusive: bool):
        with self.cv:
            if exclusive:
                self.exclusive = False
            else:
                self.shared -= 1
            self.cv.notify_all()


class Server:
    def __init__(self, hbm_budget: Optional[int] = None, max_slots: int = 32, chunk: int = 50,
                 rtol: Optional[float] = None, keep_state: bool = True, free_bytes=device_free_bytes,
                 cluster_size=cluster_ctas, precision: int = avip.PREC_MIXED):
        if hbm_budget is None:
            hbm_budget = int(free_bytes() * 0.8)
        self.budget = hbm_budget
        self.free_bytes = free_bytes  # live free device memory (a callable, replaceable in tests)
        self.cluster_size = cluster_size  # request -> CTAs of its cluster (a callable)
        self.max_slots = max_slots
        self.chunk = chunk
        self.precision = precision
        # the mixed-precision solve refines the FP64 residual to 1e-10 (its FP32 inner solve
        # cannot reach 1e-12 per refinement step); the FP64 path solves to 1e-12
        self.rtol = rtol if rtol is not None else (1e-10 if precision == avip.PREC_MIXED else 1e-12)
        self.keep_state = keep_state
        self.lock = _GpuLock()
        self.admit_log: List[tuple] = []

    def _work(self, req: Request, t0: float, release, built):
        m = None
        try:
            m = avip.Mesh(req.problem, rtol=self.rtol, pcg_kind=solver_kind(req.problem),
                          cluster_size=self.cluster_size(req.problem), precision=self.precision)
            built()  # the handle's memory is now part of what the device reports as used
            # cluster-resident solves share the GPU; whole-GPU cooperative solves run exclusively
            ex = m.info["pcg_kind"] not in CLUSTER_KINDS
            left = req.nsteps
            while left > 0:
                k = min(self.chunk, left)
                self.lock.acquire(ex)
                try:
                    st = m.run(k, allow=(avip.AVIP_OK, avip.AVIP_ENOTCONV))
                finally:
                    self.lock.release(ex)
                req.pcg_iters += st["pcg_iters_total"]
                req.status = req.status or st["status"]
                left -= k
            if self.keep_state:
                req.state = m.state()
            m.close()
        except Exception:
            req.status = avip.AVIP_ECUDA
            if m is None:
                built()
        req.done = time.perf_counter() - t0
        release()

    def run(self, requests: List[Request], realtime: bool = True) -> dict:
        """Serve the requests (arrival times relative to now).  With realtime=False every
        request is considered arrived at t = 0 (throughput mode)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        used = [0]       # estimates of the requests in service (the server's budget)
        reserved = [0]   # estimates of admitted requests whose handle is not built yet
        slots = [0]
        cv = threading.Condition()
        threads = []
        t0 = time.perf_counter()

        def release_for(req):
            def _rel():
                with cv:
                    used[0] -= estimate_bytes(req.problem)
                    slots[0] -= 1
                    cv.notify_all()
            return _rel

        def built_for(req):
            def _built():
                with cv:
                    reserved[0] -= estimate_bytes(req.problem)
                    cv.notify_all()
            return _built

        i = 0
        while i < len(pending):
            req = pending[i]
            need = estimate_bytes(req.problem)
            if need > self.budget:
                req.status = avip.AVIP_ENOMEM       # can never fit: rejected, not attempted
                req.done = req.arrival
                i += 1
                continue
            with cv:
                now = time.perf_counter() - t0
                if realtime and req.arrival > now:
                    cv.wait(timeout=req.arrival - now)
                    continue
                if slots[0] >= self.max_slots or used[0] + need > self.budget:
                    cv.wait(timeout=0.05)
                    continue
                free = self.free_bytes() - reserved[0] - FREE_MARGIN
                if need > free:
                    if slots[0] == 0 and reserved[0] == 0:  # nothing of ours to wait for: never fits
                        req.status = avip.AVIP_ENOMEM
                        req.done = req.arrival
                        i += 1
                        continue
                    cv.wait(timeout=0.05)
                    continue
                used[0] += need
                reserved[0] += need
                slots[0] += 1
                req.admitted = time.perf_counter() - t0
                self.admit_log.append((req.rid, req.admitted, used[0], free))
            th = threading.Thread(target=self._work, args=(req, t0, release_for(req), built_for(req)),
                                  daemon=True)
            th.start()
            threads.append(th)
            i += 1
        for th in threads:
            th.join()
        makespan = time.perf_counter() - t0
        return report(requests, makespan)


def run_sequential(requests: List[Request], rtol: float = 1e-12, keep_state: bool = True) -> dict:
    """The same requests one by one in arrival order on the plain FP64 path (no overlap); a
    request starts at max(its arrival, completion of the previous one)."""
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        req.admitted = time.perf_counter() - t0
        m = avip.Mesh(req.problem, rtol=rtol)
        st = m.run(req.nsteps, allow=(avip.AVIP_OK, avip.AVIP_ENOTCONV))
        req.pcg_iters = st["pcg_iters_total"]
        req.status = st["status"]
        if keep_state:
            req.state = m.state()
        m.close()
        req.done = time.perf_counter() - t0
    return report(requests, time.perf_counter() - t0)


def report(requests: List[Request], makespan: float) -> dict:
    ok = [r for r in requests if r.done >= 0 and r.status in (0, avip.AVIP_ENOTCONV)]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    cells = sum(r.problem.n_tris * r.nsteps for r in ok)
    return {"requests": len(requests), "completed": len(ok), "makespan_s": makespan,
            "cell_steps_per_s": cells / makespan if makespan > 0 else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "rejected": sum(1 for r in requests if r.status == avip.AVIP_ENOMEM)}


def poisson_requests(count: int, rate: float, seed: int, t_min: float = 5e3, t_max: float = 2e6,
                     steps_min: int = 200, steps_max: int = 5000) -> List[Request]:
    """Poisson arrivals at `rate` per second; triangle counts lognormal (median 1e5, clipped to
    [t_min, t_max]); voltage uniform in 5-25 kV; step counts uniform in [steps_min, steps_max]."""
    from . import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        T = float(np.clip(np.exp(rng.normal(np.log(1e5), 1.16)), t_min, t_max))
        volt = float(rng.uniform(5e3, 25e3))
        ar = float(rng.uniform(1.0, 4.0))
        nq = max(1.0, np.sqrt(T / (2.0 * ar)))
        nx = max(5, int(round(nq)) + 1)
        ny = max(5, int(round(nq * ar)) + 1)
        Lx = 1e-2
        p = W.plates_problem(nx, ny, Lx, Lx * (ny - 1) / (nx - 1), volt, seed=seed * 7919 + k,
                             field_dependent=True, source=W.SRC_TOWNSEND, name=f"req{k}")
        steps = int(rng.integers(steps_min, steps_max + 1))
        out.append(Request(k, t, p, steps))
    return out
