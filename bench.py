"""Throughput of the Poisson-coupled drift-diffusion step on GB300 (cell-steps/s).

Default workload: the pin-plane streamer, 1 cm x 2 cm, 500 x 1000 jittered nodes (997,002
triangles), Morton-ordered, 20 kV needle anode, local-field electron mobility mu ~ E^-0.2,
Townsend ionisation, plain FP64, CG rtol 1e-12.  One step = Poisson (CG preconditioned by an
AMG V-cycle to rtol, warm-started; `--pcg-kind 2` for Jacobi-PCG) + E + gradients + time step +
fluxes + source + update, all in the CUDA library.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun with one independent replica per GPU (weak scaling; the path has no
data exchange).  `--impl reference` times the FP64 CPU oracle on the host cores instead.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s (DD+Poisson) plain vs mixed/batched/served; p50/p99 latency"
UNIT = "cell-steps/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 data-sheet rate, used only if the in-run probe fails


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pin_plane", choices=["pin_plane", "pin_plane_hybrid", "hyperbole_ml", "plates65", "axisym",
                                                            "axisym_photo", "batch256", "served", "sweep"])
    ap.add_argument("--instances", type=int, default=256, help="batch256: number of instances")
    ap.add_argument("--requests", type=int, default=24, help="served: number of requests in the sample")
    ap.add_argument("--req-steps", type=int, nargs=2, default=[20, 60], help="served: step-count range")
    ap.add_argument("--served-fp64", action="store_true", help="served: serve on the FP64 path (default mixed)")
    ap.add_argument("--rtol", type=float, default=1e-12)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="mixed = FP32 inner PCG with FP64 refinement of the Poisson residual")
    ap.add_argument("--scheme", default="llw", choices=["llw", "sg"],
                    help="edge flux: limited Lax-Wendroff (default) or Scharfetter-Gummel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true", help="skip nvidia-smi sampling (diagnosis only)")
    ap.add_argument("--pcg-threads", type=int, default=0, help="PCG block size (0 = library default)")
    ap.add_argument("--pcg-kind", type=int, default=0,
                    help="solver kernel: 0 auto, 1 streaming, 2 register-resident, 5 cluster-resident, 7 BiCGStab, "
                         "8 AMG-preconditioned CG")
    ap.add_argument("--precond-fp64", action="store_true",
                    help="AMG solvers: apply the V-cycle in FP64 instead of FP32")
    ap.add_argument("--pcg-max-iter", type=int, default=0,
                    help="cap PCG iterations per solve (profiling captures only; not a bench setting)")
    return ap.parse_args()


def make_problem(name, scheme="llw"):
    p, desc = _make_problem(name)
    if scheme == "sg":
        from paper_2201_01291_gb300 import workloads as W
        p.opts.scheme = W.FLUX_SG
        desc += ", Scharfetter-Gummel edge flux"
    return p, desc


def _make_problem(name):
    from paper_2201_01291_gb300 import workloads as W
    if name == "pin_plane":
        p = W.config_pin_plane()
        desc = ("pin-plane streamer 1cm x 2cm, 500x1000 jittered nodes (997,002 tris), Morton order, "
                "20 kV needle, mu_e ~ E^-0.2, Townsend alpha (air-like, 1 atm), e + positive ions, FP64")
    elif name == "pin_plane_hybrid":
        p = W.config_pin_plane_hybrid()
        desc = (f"pin-plane streamer 1cm x 2cm on a hybrid mesh, 500x1000 jittered nodes, {p.quads.shape[0]:,} "
                f"quadrangles + {p.n_tris:,} triangles (each grid cell a quadrangle with probability 0.5), "
                "Morton order, 20 kV needle, mu_e ~ E^-0.2, Townsend alpha, e + positive ions, FP64")
    elif name == "hyperbole_ml":
        p = W.config_hyperbole_ml()
        desc = ("three-species air chemistry (ionisation, attachment, e-p and n-p recombination, immobile "
                "ions) at 1000 K, 5mm x 5mm gap, 800x800 jittered nodes (1,278,402 tris), 1 mm needle anode "
                "ramped 0 -> 5 kV in 2 ns, 1e15 m^-3 background, Morton order, FP64")
    elif name == "axisym_photo":
        p = W.config_axisym_photo()
        desc = ("axisymmetric (x, r) streamer gap 1.25cm x 1.25cm, 701x701 jittered nodes (980,000 tris), "
                "1e9 m^-3 background, photoionisation by the three-term Helmholtz fit (three extra solves per "
                "step, AMG-preconditioned BiCGStab each), 18.75 kV, mu_e ~ E^-0.2, Townsend alpha, FP64")
    elif name == "axisym":
        p = W.config_axisym_streamer()
        desc = ("axisymmetric (x, r) streamer gap 1.25cm x 1.25cm, 701x701 jittered nodes (980,000 tris), "
                "Morton order, 18.75 kV (1.5 MV/m), seed 5e18 m^-3 on the axis at x = 1 cm, mu_e ~ E^-0.2, "
                "Townsend alpha, e + positive ions, r-weighted Poisson solved by BiCGStab, FP64")
    else:
        p = W.config_plates_65()
        desc = "parallel plates 1cm x 1cm, 65x65 jittered nodes (8192 tris), 5 kV, constant mu/D, FP64"
    return p, desc


def workload_config(problem, desc, args):
    """The `config` dict of the JSON line: the workload only, identical in both arms."""
    return {"workload": desc, "n_nodes": int(problem.n_nodes), "n_cells": int(problem.n_cells),
            "rtol": args.rtol, "precision": args.precision, "seed": problem.seed}


def host_cpu():
    """CPU model and the number of cores visible to this process."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count()
    return {"cpu_model": model or "unknown", "nproc": n}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "500"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (driver/NVML initialisation) can stall the GPU's work
            # submission for a few hundred ms: let it finish before the timed region starts
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(elapsed, units_per_rank, world, device="cuda"):
    """Whole-job figures of a replicated run: the slowest rank's elapsed time (max over ranks)
    and the units of all ranks divided by it."""
    if world > 1:
        import torch
        t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
    return elapsed, world * units_per_rank / elapsed


KERNEL_NAMES = {1: "pcg_fp64_kernel (streaming)", 2: "pcg_fp64_res_kernel (register-resident)",
                4: "pcg_mixed_kernel (FP32 inner + FP64 refinement)", 5: "pcg_cluster_kernel (cluster-resident)",
                7: "bicgstab_fp64_kernel (non-symmetric, axisymmetric)",
                8: "pcg_amg_kernel (CG + smoothed-aggregation AMG V-cycle)",
                9: "bicgstab_amg_kernel (BiCGStab + AMG V-cycle, axisymmetric)",
                10: "pcg_amg_mixed_kernel (FP32 CG + FP32 AMG V-cycle, FP64 refinement)",
                11: "pcg_amg_cluster_kernel (AMG-preconditioned CG on one cluster)"}

# DRAM bytes per solver iteration measured by ncu on the pin-plane 500 x 1000 workload (the
# counters of one captured launch divided by its iterations), keyed by solver kind; valid for the
# kernel revision the capture was taken on and for that workload only.
NCU_DRAM_BYTES_PER_ITER = {
    # pcg_fp64_res_kernel: 300-iteration capture, L2-resident working set
    2: ((72.372224e6 + 2.023936e6) / 300.0, "ncu DRAM read+write of a 300-iteration capture scaled to the "
                                            "launch's iterations (L2-resident working set)"),
    # pcg_amg_kernel<1024, float>: one 21-iteration solve (two-phase V-cycle, Jacobi smoother,
    # spill-free streams)
    8: ((3574.051e6 + 28.363e6) / 21.0, "ncu DRAM read+write of a 21-iteration solve scaled to the launch's "
                                        "iterations (profiles/pcg_amg_kernel_pin_plane_500x1000.md)"),
}


def pcg_traffic_model(info, iters, solves):
    """Algorithmic bytes and flops of one step's PCG launch, per the kernel that runs:
    streaming (1): per iteration 12 B per stored entry (int32 column + FP64 value) + 4 B row
        length + r gather 8 + p, q read/write 32 (phase A) + x, r read/write 32, p, q reads 16
        (phase B) = 12 nnz + 92 N bytes;
    register-resident (2): p, q, x in registers: 12 nnz + r gather 8 + r read/write 16
        = 12 nnz + 24 N bytes;
    mixed (4): FP32 inner iteration 8 nnz + 48 N bytes (FP64 outer residuals not counted);
    flops: 2 nnz + 12 N per iteration (SpMV, 3 recurrences, 2 dots, x update);
    BiCGStab (7): two gathers per iteration, 12 B per stored entry each; phase S gathers v
        (8 + 4 B row length), reads r, A r, rh (24), writes z, s, t (24); phase R gathers t
        (8 + 4), reads s, p, v, z, rh, x (48), writes x, r, A r, p, v (40): 24 nnz + 160 N bytes;
        flops 4 nnz + 32 N per iteration."""
    N, nnz, kind = info["n_nodes"], info["nnz"], info["pcg_kind"]
    if kind in (8, 9, 10):
        return amg_traffic_model(info["levels"], nnz, N, iters, solves, kind, sv=info.get("precond_bytes", 4))
    per_it = {1: 12 * nnz + 92 * N, 2: 12 * nnz + 24 * N, 4: 8 * nnz + 48 * N, 7: 24 * nnz + 160 * N}.get(kind, 0)
    # per solve: the set-up (the cubic predictor reads four potentials and shifts three, the
    # right-hand side) and the final true residual
    per_solve = {1: 24 * nnz + 116 * N, 2: 24 * nnz + 96 * N, 4: 24 * nnz + 116 * N,
                 7: 24 * nnz + 186 * N}.get(kind, 0)
    bytes_ = iters * per_it + solves * per_solve
    if kind == 7:
        flops = iters * (4 * nnz + 32 * N) + solves * (4 * nnz + 20 * N)
    else:
        flops = iters * (2 * nnz + 12 * N) + solves * (4 * nnz + 12 * N)
    return bytes_, flops


def amg_traffic_model(levels, nnz0, N, iters, solves, kind=8, sv=4):
    """Algorithmic bytes and flops of one step's AMG-preconditioned launch (kinds 8, 9, 10).

    Conventions: every stored entry of an operator is read once (4 B column + sv B value; sv = 4
    for the FP32 hierarchy, 8 for FP64) and costs 2 flops; a gathered vector is read once per
    product (as if every reuse hit a cache), an own-row element once per access, a written
    element once.  With levels[l] = (n, nnz A, nnz P, nnz Rf, nnz U, nnz Pf) and n' the next
    level's rows, one V-cycle moves, per non-coarsest level:
      down  rf (4 + sv) + sv (4 n + n')      [Rf b gathers b; xp = Q b elementwise: b, Q's
                                              diagonal read, xp written; b' written]
      up    (u + pf)(4 + sv) + sv (2 n + n') [[U | Pf] [xp; x'] gathers xp and x'; x written]
    and on the coarsest level sv (n_c^2 + 2 n_c) (dense inverse, b read, x written).  In the FP64
    CG (kind 8) the finest down phase gathers FP32 copies of r and q (2 sv N in place of sv N for
    b), reads r, q, x, p and writes r, x and the copy of r (32 + 16 + sv bytes per row); the finest
    up phase reads r and writes z in FP64 (8 + 8 - sv N more); w = A z reads A (12 nnz), gathers
    z (8 N), reads z, q, p (24 N), writes q, p and q's copy (16 + sv N).  BiCGStab (kind 9)
    applies two V-cycles per iteration with FP64 input and output (8 - sv more per row at each
    end) and its phases add 24 nnz + 216 N bytes.  The mixed-precision solve (kind 10) runs the
    FP32 V-cycle on FP32 vectors and its inner CG moves 8 B per stored entry of A and 4 B per
    vector element: 8 nnz + 60 N.  Per solve: set-up (the cubic predictor reads four potentials
    and shifts three) and the final true residual, 24 nnz + 116 N.
    Flops (returned: FP64 operations only, the unit the FP64 roofline compares): 2 per stored
    entry of every FP64 product and per-row vector operations; the V-cycle's own 2 per stored
    entry and 2 per row and level count only with an FP64 hierarchy (sv = 8)."""
    vb, vf = 0.0, 0.0
    nl = len(levels)
    for l, (n, a, p, rf, u, pf) in enumerate(levels):
        if l + 1 < nl:
            nn = levels[l + 1][0]
            vb += rf * (4 + sv) + sv * (4 * n + nn)
            vb += (u + pf) * (4 + sv) + sv * (2 * n + nn)
            vf += 2 * (rf + u + pf) + 2 * n
        else:
            vb += sv * (n * n + 2 * n)
            vf += 2 * n * n
    if sv != 8:
        vf = 0.0  # the V-cycle runs in FP32
    if kind == 9:
        per_it = 2 * (vb + 2 * (8 - sv) * N) + 24 * nnz0 + 216 * N
        fl_it = 2 * vf + 4 * nnz0 + 32 * N
    elif kind == 10:
        per_it = vb + 8 * nnz0 + 60 * N
        fl_it = 0.0  # FP32 inner solve; the few FP64 outer residuals are counted per solve
    else:
        per_it = (vb + sv * N + (48 + sv) * N + (16 - sv) * N
                  + 12 * nnz0 + 8 * N + 24 * N + (16 + sv) * N)
        fl_it = vf + 2 * nnz0 + 14 * N
    per_solve = 24 * nnz0 + 116 * N
    return iters * per_it + solves * per_solve, iters * fl_it + solves * (4 * nnz0 + 12 * N)


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2201_01291_gb300 import build, avip
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
        build.build()
    avip.load()
    problem, desc = make_problem(args.workload, args.scheme)
    T = problem.n_cells
    stream = torch.cuda.Stream()
    kw = {"max_iter": args.pcg_max_iter} if args.pcg_max_iter > 0 else {}
    allow = (avip.AVIP_OK, avip.AVIP_ENOTCONV) if args.pcg_max_iter > 0 else (avip.AVIP_OK,)
    prec = avip.PREC_MIXED if args.precision == "mixed" else avip.PREC_FP64
    kw["precond_fp64"] = 1 if args.precond_fp64 else 0
    m = avip.Mesh(problem, rtol=args.rtol, stream=stream.cuda_stream, pcg_threads=args.pcg_threads,
                  pcg_kind=args.pcg_kind, precision=prec, **kw)
    # roofline denominators of this device, measured now (before the timed region)
    rc64, fp64_peak = avip.peak_probe(avip.PROBE_FP64_FMA, stream.cuda_stream)
    rcbw, copy_gbs = avip.peak_probe(avip.PROBE_HBM_COPY, stream.cuda_stream)
    torch.cuda.synchronize()
    # warm-up (graph capture happens here too)
    with torch.cuda.stream(stream):
        m.run(args.warmup, allow=allow)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank) if rank == 0 and not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    kernel_ms = dict.fromkeys(avip.TIMED_KERNELS, 0.0)
    iters = 0
    launches = 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        # K steps queued back to back with events around every kernel, one wait at the end; the
        # working set moved per step (the solver's operators alone stream ~2 GB) is far larger
        # than L2, so no step finds the previous one's data cached
        ev0.record(stream)
        ms, st = m.run_timed(args.steps, allow=allow)
        ev1.record(stream)
    torch.cuda.synchronize()
    for key in kernel_ms:
        kernel_ms[key] += ms[key]
    iters += st["pcg_iters_total"]
    photo = m.photo_stats() if problem.photo is not None else None
    # per step: pcg, node_fields, dt_cells, (edge_flux in FP64,) flux_update, finalize; photoionisation:
    # the solves (one launch side by side, else one per term) and the source update
    n_photo = 0 if photo is None else (1 if photo["side_by_side"] else len(problem.photo.a)) + 1
    # plus one statistics reset per call (memsets are not kernels and are not counted)
    launches += 1 + args.steps * (5 + (1 if args.precision == "fp64" else 0) + n_photo)
    if world > 1:
        torch.distributed.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clocks = sampler.stop() if sampler else None
    elapsed, value = aggregate(elapsed, T * args.steps, world)
    # ---- end to end through the public API with host buffers
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 10))
    # the state lives in pinned host memory: each step uploads it and reads the new one back
    host = torch.empty(m.state().size, dtype=torch.float64, pin_memory=True).numpy()
    m.state(out=host)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m.set_state(host)
        m.run(1, allow=allow)
        m.state(out=host)
    e2e_t, _ = aggregate(max(time.perf_counter() - t0, 1e-9), 1, world)
    state_bytes = host.size * 8
    info = dict(m.info, precond_bytes=8 if (args.precond_fp64 and args.precision == "fp64") else 4)
    m.close()
    # a fresh handle for the oracle comparison of the CPU-baseline leg (same steps from t = 0)
    check = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mc = avip.Mesh(problem, rtol=args.rtol, pcg_kind=args.pcg_kind, precision=prec, **kw)
        with torch.cuda.stream(stream):
            mc.run(args.cpu_steps, allow=allow)
        torch.cuda.synchronize()
        check = ([mc.density(s) for s in range(len(problem.species))], mc.phi())
        mc.close()
    if rank != 0:
        return None
    # ---- roofline of the dominant kernel (PCG)
    peaks = measured_peaks()
    kernel_name = KERNEL_NAMES.get(info["pcg_kind"], str(info["pcg_kind"]))
    if info["pcg_kind"] == 11:  # the one-cluster AMG solve moves the bytes of kind 8 or 10
        info = dict(info, pcg_kind=10 if args.precision == "mixed" else 8)
    byts, flops = pcg_traffic_model(info, iters, args.steps)
    pcg_s = kernel_ms["pcg"] / 1e3
    hbm = peaks.get("hbm_gbs")
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    if not hbm:
        hbm, hbm_src = (copy_gbs, "measured in this run (copy probe)") if rcbw == 0 else (6800.0, "fallback")
    if rc64 == 0 and fp64_peak > 0:
        f64, f64_src = fp64_peak, "measured in this run (FP64 FMA-chain probe, peak_probe)"
    else:
        f64, f64_src = FP64_NOMINAL_TFLOPS, "nominal (the in-run probe failed)"
    gbs = byts / pcg_s / 1e9
    tfl = flops / pcg_s / 1e12
    kind = info["pcg_kind"]
    # the binding roof is the unit the kernel uses the largest fraction of; the FP32 inner
    # solve of the mixed path is compared with HBM only (its FP32 rate is far from binding)
    hbm_frac, f64_frac = gbs / hbm, tfl / f64
    if kind in (4, 10) or hbm_frac >= f64_frac:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(hbm_frac, 4), "peak_source": hbm_src}
    else:
        roof = {"bound": "alu", "achieved": round(tfl, 4), "peak": round(f64, 4), "unit": "TFLOP/s",
                "frac": round(f64_frac, 4), "peak_source": f64_src}
    roof.update({"hbm_gbs_algorithmic": round(gbs, 1), "hbm_frac_of_measured": round(hbm_frac, 4),
                 "fp64_tflops": round(tfl, 4), "fp64_frac_of_measured": round(f64_frac, 4),
                 "fp64_peak_tflops_measured": round(fp64_peak, 4) if rc64 == 0 else None,
                 "copy_gbs_measured_in_run": round(copy_gbs, 1) if rcbw == 0 else None})
    per_launch_iters = iters / args.steps
    traffic, note = NCU_DRAM_BYTES_PER_ITER.get(kind, (None, None)) if args.workload == "pin_plane" else (None, None)
    roof.update({"kernel": kernel_name,
                 "traffic": int(traffic * per_launch_iters) if traffic else None,
                 "traffic_note": note,
                 "algorithmic_bytes_per_launch": int(byts / args.steps),
                 "pcg_iters_per_step": per_launch_iters,
                 "kernel_ms_per_step": {k: round(v / args.steps, 4) for k, v in kernel_ms.items()}})
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": workload_config(problem, desc, args),
        "preconditioner": ("AMG V-cycle in " + ("FP64" if info["precond_bytes"] == 8 else "FP32") +
                           "; Krylov iterate, residuals, products with the Poisson matrix and stopping test in FP64")
        if info["pcg_kind"] in (8, 9, 11) else None,
        "parallelism": f"replicas x{world}", "nnz": info["nnz"],
        "l2": "working set per step far larger than L2 (the solver streams ~2 GB of operators per step); no flush",
        "e2e": {"value": world * T * e2e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes,
                "how": "per step: state_set from pinned host memory, run_steps(1), state_get to pinned host memory"},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
    }
    if photo is not None:
        out["photoionisation"] = {"solves": "side by side in one launch" if photo["side_by_side"] else "one by one",
                                  "iters_last_step": photo["iters"],
                                  "ms_per_step": round(kernel_ms["photo"] / args.steps, 4)}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], ref = cpu_baseline(problem, args.cpu_steps)
        n_gpu, phi_gpu = check
        err = {"steps": args.cpu_steps, "phi": normwise(phi_gpu, ref[1])}
        for s_, sp_ in enumerate(problem.species):
            err["n_" + str(s_)] = normwise(n_gpu[s_], ref[0][s_])
        err["max"] = max(v for k, v in err.items() if k != "steps")
        err["metric"] = "norm-wise max_i |x - x_oracle| / max_i |x_oracle|, fresh handle vs the CPU-baseline oracle run"
        out["oracle_error"] = err
    return out


def normwise(x, ref):
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(x - ref).max() / scale) if scale > 0 else float(np.abs(x).max())


def run_batch(args, rank, world, local_rank):
    """Many uneven instances advanced together (one persistent cluster PCG launch per step for
    all instances + batched drift-diffusion stages, CUDA-graph replay, autotuned cluster size).
    Instances: triangles log-uniform in [2e3, 2e5], aspect 1-4, 5-25 kV, 2 or 3 species."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2201_01291_gb300 import build, avip, workloads as W
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    avip.load()
    t0 = time.perf_counter()
    probs = W.random_instances(args.instances, seed=4 + 1000 * rank)
    prec = avip.PREC_MIXED if args.precision == "mixed" else avip.PREC_FP64
    # instances above 2,000 nodes solve with the cluster form of the AMG-preconditioned CG (kind 8,
    # or kind 10 in mixed precision); the smaller ones with the shared-memory Jacobi-PCG
    meshes = [avip.Mesh(p, rtol=args.rtol, precision=prec,
                        pcg_kind=(8 if prec == avip.PREC_FP64 else 10) if p.n_nodes > 2000 else 0) for p in probs]
    b = avip.Batch(meshes, cluster_size=0)
    setup = time.perf_counter() - t0
    T = sum(p.n_tris for p in probs)
    b.run(args.warmup)
    sampler = ClockSampler(local_rank) if rank == 0 and not args.no_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st = b.run(args.steps)          # graph replays; the call returns after the device finished
    elapsed = time.perf_counter() - t1
    clocks = sampler.stop() if sampler else None
    elapsed, _ = aggregate(elapsed, 1, world)
    iters = sum(x["pcg_iters_total"] for x in st)
    # end to end: per step every instance's state in from host, one batch step, state back
    e2e_steps = 0 if args.no_e2e else 2
    # every instance's state in one pinned host buffer, moved by the batch checkpoint calls
    host = torch.empty(b.state_size(), dtype=torch.float64, pin_memory=True).numpy()
    b.state(out=host)
    t2 = time.perf_counter()
    for _ in range(e2e_steps):
        b.set_state(host)
        b.run(1)
        b.state(out=host)
    e2e_t = max(time.perf_counter() - t2, 1e-9)
    state_bytes = host.size * 8
    info = dict(b.info)
    b.close()
    for m in meshes:
        m.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": world * T * args.steps / elapsed, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"batched: {args.instances} instances, triangles log-uniform in [2e3, 2e5] "
                               f"(total {T}), aspect 1-4, 5-25 kV, 2 or 3 species, {args.precision}",
                   "instances": args.instances, "n_tris_total": T, "rtol": args.rtol, "precision": args.precision,
                   "cluster": info, "setup_s": round(setup, 1), "parallelism": f"replicas x{world}",
                   "l2": "working set larger than L2", "timing": "host clock around synchronous graph replays"},
        "pcg_iters_per_step": iters / args.steps,
        "e2e": {"value": world * T * e2e_steps / e2e_t if e2e_steps else None, "unit": UNIT,
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
        "gpu_launches": 1 + 5 * args.steps,  # statistics reset, then per step the solve and 4 stages
        "clocks": clocks,
    }


def run_served(args, rank, world, local_rank):
    """Poisson arrivals at 50 requests/s of discharge solves (triangles lognormal, median 1e5,
    clipped to [5e3, 2e6]; 5-25 kV; steps uniform in --req-steps), served with continuous
    batching (admission by free HBM, resident state, overlapping work) in mixed precision
    (within 1e-6 of the FP64 oracle), against the same requests run one by one on the plain
    FP64 path."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2201_01291_gb300 import build, avip, serve
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    avip.load()
    lo, hi = args.req_steps
    reqs = serve.poisson_requests(args.requests, 50.0, seed=5 + 1000 * rank, steps_min=lo, steps_max=hi)
    # warm-up: compile paths, first-touch
    warm = serve.poisson_requests(2, 50.0, seed=999, t_max=2e4, steps_min=5, steps_max=5)
    serve.Server(keep_state=False, precision=avip.PREC_FP64 if args.served_fp64 else avip.PREC_MIXED).run(
        warm, realtime=False)
    sampler = ClockSampler(local_rank) if rank == 0 and not args.no_clocks else None
    if sampler:
        sampler.start()
    prec = avip.PREC_FP64 if args.served_fp64 else avip.PREC_MIXED
    srv = serve.Server(chunk=25, keep_state=False, precision=prec)
    served = srv.run(reqs)
    clocks = sampler.stop() if sampler else None
    seq_reqs = serve.poisson_requests(args.requests, 50.0, seed=5 + 1000 * rank, steps_min=lo, steps_max=hi)
    seq = serve.run_sequential(seq_reqs, keep_state=False)
    if rank != 0:
        return None
    T = sum(r.problem.n_tris for r in reqs)
    return {
        "metric": METRIC, "value": served["cell_steps_per_s"] * world, "unit": UNIT, "n_gpus": world,
        "steps": sum(r.nsteps for r in reqs), "warmup": 1, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.served_fp64 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"served: {args.requests} Poisson arrivals at 50 req/s, triangles lognormal "
                               f"(median 1e5, clipped to [5e3, 2e6]; this sample {T} in total), 5-25 kV, "
                               f"steps uniform in [{lo}, {hi}], " + ("FP64" if args.served_fp64 else "mixed precision"),
                   "requests": args.requests,
                   "precision": "fp64" if args.served_fp64 else "mixed (FP32 solve and fluxes, FP64 refinement "
                   "and state)", "parallelism": f"replicas x{world}"},
        "served": served, "sequential_fp64": seq,
        "p50_latency_s": served["p50_latency_s"], "p99_latency_s": served["p99_latency_s"],
        "e2e": {"value": served["cell_steps_per_s"] * world, "unit": UNIT,
                "how": "requests from host problem descriptions to host results, wall clock"},
        "clocks": clocks,
    }


def run_sweep(args, rank, world, local_rank):
    """PCG throughput across mesh sizes, from L2-resident to far past L2 (pin-plane shape,
    1 cm x 2 cm, FP64): per size the kernel chosen by the library, iterations, us per
    iteration, algorithmic GB/s and FP64 TFLOP/s against the peaks."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2201_01291_gb300 import build, avip, workloads as W
    build.build()
    avip.load()
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    rows = []
    for nx in (160, 320, 500, 1000, 1415, 2000):
        ny = 2 * nx
        p = W.plates_problem(nx, ny, 1e-2, 2e-2, 2e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND,
                             needle_len=2e-3)
        m = avip.Mesh(p, rtol=args.rtol, pcg_kind=args.pcg_kind)
        m.run(2)
        ms, st = m.run_timed(2)
        info = m.info
        m.close()
        it = st["pcg_iters_total"]
        byts, flops = pcg_traffic_model(info, it, 2)
        s_ = ms["pcg"] / 1e3
        rows.append({"n_nodes": info["n_nodes"], "n_tris": info["n_tris"], "kernel": KERNEL_NAMES.get(info["pcg_kind"]),
                     "iters_per_step": it / 2, "us_per_iter": 1e6 * s_ / it,
                     "gbs": round(byts / s_ / 1e9, 1), "hbm_frac": round(byts / s_ / 1e9 / hbm, 3),
                     "fp64_tflops": round(flops / s_ / 1e12, 3),
                     "cell_steps_per_s": p.n_tris * 2 / (sum(ms.values()) / 1e3)})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    if rank != 0:
        return None
    return {"metric": METRIC, "workload": "size sweep (PCG roofline)", "rows": rows, "unit": UNIT}


def oracle_module():
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import avip_oracle
    return avip_oracle


def cpu_baseline(problem, steps):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload.
    Returns the baseline record and the oracle's densities and potential after `steps` steps
    from the initial state (the reference of the line's oracle_error)."""
    O = oracle_module()
    t0 = time.perf_counter()
    o = O.Oracle(problem)
    setup = time.perf_counter() - t0
    n = o.initial_state()
    t1 = time.perf_counter()
    c1 = time.process_time()
    t = 0.0
    phi = None
    for _ in range(steps):
        n, info = o.step(n, t=t)
        t += info["dt"]
        phi = info["phi"]
    wall = time.perf_counter() - t1
    cpu = time.process_time() - c1
    hc = host_cpu()
    rec = {"value": problem.n_cells * steps / wall, "unit": UNIT, "cores": max(1, round(cpu / wall)),
           "kind": "oracle", "cpu_model": hc["cpu_model"], "nproc": hc["nproc"],
           "sample": f"{steps} explicit steps of the same workload after a {setup:.1f} s one-off "
                     f"setup (metrics + sparse LU factorisation, excluded); numpy/scipy"}
    return rec, (n, phi)


def run_reference(args, rank, world):
    if rank != 0:
        return None
    problem, desc = make_problem(args.workload, args.scheme)
    O = oracle_module()
    t0 = time.perf_counter()
    o = O.Oracle(problem)
    setup = time.perf_counter() - t0
    n = o.initial_state()
    for _ in range(args.warmup):
        n, _ = o.step(n)
    c1 = time.process_time()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        n, _ = o.step(n)
    wall = time.perf_counter() - t1
    cpu = time.process_time() - c1
    value = problem.n_cells * args.steps / wall
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(problem, desc, args), "parallelism": "cpu oracle (rank 0 only)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(1, round(cpu / wall)), "kind": "oracle",
                             **host_cpu(),
                             "sample": f"each step one explicit oracle step of the workload "
                                       f"(setup {setup:.1f} s excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        fn = {"batch256": run_batch, "served": run_served, "sweep": run_sweep}.get(args.workload, run_ours)
        out = fn(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
