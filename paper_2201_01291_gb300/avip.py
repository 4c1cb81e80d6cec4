"""Thin Python binding of the C ABI in include/avip.h (argument marshalling only).

Every function of the header is exposed under the same name; `Mesh` is a convenience wrapper
that creates a handle from a synthetic workload description and owns it.  All computation
runs in the CUDA library; if the library is missing or cannot be loaded the import fails
loudly (there is no CPU path).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libavip.so")

AVIP_OK, AVIP_EINVAL, AVIP_ENOMEM, AVIP_ENOTCONV, AVIP_ENAN, AVIP_ECUDA, AVIP_ETIMEOUT, AVIP_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
FIELD_PHI, FIELD_EX, FIELD_EY, FIELD_DENSITY, FIELD_VOLUME, FIELD_PHOTO = 0, 1, 2, 3, 4, 5
MAX_PHOTO_TERMS = 3
PREC_FP64, PREC_MIXED = 0, 1
GEOM_PLANAR, GEOM_AXISYMMETRIC = 0, 1
FLUX_LLW, FLUX_SG = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class AvipOpts(C.Structure):
    _fields_ = [("cfl", C.c_double), ("fourier", C.c_double), ("a_diel", C.c_double), ("a_chem", C.c_double),
                ("beta", C.c_double), ("limiter", C.c_int32), ("precision", C.c_int32), ("rtol", C.c_double),
                ("max_iter", C.c_int32), ("reorder", C.c_int32), ("dt_fixed", C.c_double),
                ("inner_rtol", C.c_double), ("pcg_threads", C.c_int32), ("pcg_kind", C.c_int32),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("geometry", C.c_int32), ("scheme", C.c_int32),
                ("v_rise", C.c_double), ("wait_timeout", C.c_double), ("precond_fp64", C.c_int32),
                ("cluster_size", C.c_int32)]


class AvipStats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("pcg_iters_total", C.c_int32), ("pcg_iters_max", C.c_int32),
                ("status", C.c_int32), ("dt_min", C.c_double), ("dt_max", C.c_double), ("t", C.c_double),
                ("charge", C.c_double), ("charge_start", C.c_double), ("relres_max", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AvipError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} ({code}) {last_error()}")


_P = C.POINTER
_D = _P(C.c_double)
_I = _P(C.c_int32)
_H = C.c_void_p

_SIGS = {
    "avip_opts_default": (C.c_int, [_P(AvipOpts)]),
    "mesh_create": (C.c_int, [_D, C.c_int32, _I, C.c_int32, _I, _D, _P(AvipOpts), _P(_H)]),
    "mesh_create_hybrid": (C.c_int, [_D, C.c_int32, _I, C.c_int32, _I, C.c_int32, _I, _D, _P(AvipOpts), _P(_H)]),
    "mesh_destroy": (C.c_int, [_H]),
    "mesh_inspect": (C.c_int, [_D, C.c_int32, _I, C.c_int32, _I, C.c_int32, _I, _D, C.c_int32, _P(C.c_int64),
                               _D, _I, _D, _D]),
    "avip_inspect_error": (C.c_char_p, []),
    "mesh_set_stream": (C.c_int, [_H, C.c_void_p]),
    "mesh_set_wait_timeout": (C.c_int, [_H, C.c_double]),
    "mesh_info": (C.c_int, [_H, _P(C.c_int64)]),
    "solver_levels": (C.c_int, [_H, _P(C.c_int64), C.c_int32]),
    "species_set": (C.c_int, [_H, C.c_int32, C.c_int32, C.c_int32, _D, C.c_double, C.c_int32, _D]),
    "source_set": (C.c_int, [_H, C.c_int32, _D, _I]),
    "photo_set": (C.c_int, [_H, C.c_int32, _D, _D, C.c_double]),
    "photo_stats": (C.c_int, [_H, _I, _I, _D, _I]),
    "poisson_solve": (C.c_int, [_H, _I, _D]),
    "dd_step": (C.c_int, [_H, C.c_double, _D]),
    "run_steps": (C.c_int, [_H, C.c_int32, _P(AvipStats)]),
    "run_steps_timed": (C.c_int, [_H, C.c_int32, _D, _P(AvipStats)]),
    "field_get": (C.c_int, [_H, C.c_int32, C.c_int32, _D]),
    "state_size": (C.c_int, [_H, _P(C.c_int64)]),
    "state_get": (C.c_int, [_H, _D]),
    "state_set": (C.c_int, [_H, _D]),
    "batch_create": (C.c_int, [_P(_H), C.c_int32, C.c_int32, _P(_H)]),
    "batch_run_steps": (C.c_int, [_H, C.c_int32, C.c_void_p]),
    "batch_info": (C.c_int, [_H, _P(C.c_int64)]),
    "batch_set_dd_threads": (C.c_int, [_H, C.c_int32]),
    "batch_state_get": (C.c_int, [_H, _D]),
    "batch_state_set": (C.c_int, [_H, _D]),
    "batch_destroy": (C.c_int, [_H]),
    "pcg_csr_static": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_double, C.c_int32, C.c_void_p, _I, _D]),
    "peak_probe": (C.c_int, [C.c_int32, C.c_void_p, _D]),
    "fp64_math_check": (C.c_int, [_D]),
    "avip_status_str": (C.c_char_p, [C.c_int]),
    "avip_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: Optional[str] = None):
    """Load the shared library (build it first with paper_2201_01291_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2201_01291_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def status_str(code: int) -> str:
    return load().avip_status_str(code).decode()


def last_error() -> str:
    return load().avip_last_error().decode()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_I)


def _check(rc, where, ok=(AVIP_OK,)):
    if rc not in ok:
        raise AvipError(rc, where)
    return rc


# ------------------------------------------------------------------ same names as the C ABI
def avip_opts_default() -> AvipOpts:
    o = AvipOpts()
    _check(load().avip_opts_default(C.byref(o)), "avip_opts_default")
    return o


def mesh_create(xy, tris, node_bc, phi_D, opts: AvipOpts):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1)
    node_bc = np.ascontiguousarray(node_bc, dtype=np.int32)
    phi_D = np.ascontiguousarray(phi_D, dtype=np.float64)
    h = _H()
    rc = load().mesh_create(_dptr(xy), xy.size // 2, _iptr(tris), tris.size // 3, _iptr(node_bc), _dptr(phi_D),
                            C.byref(opts), C.byref(h))
    return rc, h


def mesh_create_hybrid(xy, tris, quads, node_bc, phi_D, opts: AvipOpts):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    tris = np.ascontiguousarray(tris if tris is not None else np.zeros(0), dtype=np.int32).reshape(-1)
    quads = np.ascontiguousarray(quads if quads is not None else np.zeros(0), dtype=np.int32).reshape(-1)
    node_bc = np.ascontiguousarray(node_bc, dtype=np.int32)
    phi_D = np.ascontiguousarray(phi_D, dtype=np.float64)
    h = _H()
    rc = load().mesh_create_hybrid(_dptr(xy), xy.size // 2, _iptr(tris) if tris.size else None, tris.size // 3,
                                   _iptr(quads) if quads.size else None, quads.size // 4, _iptr(node_bc),
                                   _dptr(phi_D), C.byref(opts), C.byref(h))
    return rc, h


def mesh_inspect(xy, tris, quads, node_bc, phi_D, geometry=0):
    """Host-only metrics of the prepared mesh (no device): dict with vol, edges, S_edge, S_b,
    nnz and n_cells in the caller's numbering."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    tris = np.ascontiguousarray(tris if tris is not None else np.zeros(0), dtype=np.int32).reshape(-1)
    quads = np.ascontiguousarray(quads if quads is not None else np.zeros(0), dtype=np.int32).reshape(-1)
    node_bc = np.ascontiguousarray(node_bc, dtype=np.int32)
    phi_D = np.ascontiguousarray(phi_D, dtype=np.float64)
    n = xy.size // 2
    counts = np.zeros(3, dtype=np.int64)
    args = (_dptr(xy), n, _iptr(tris) if tris.size else None, tris.size // 3, _iptr(quads) if quads.size else None,
            quads.size // 4, _iptr(node_bc), _dptr(phi_D), int(geometry), counts.ctypes.data_as(_P(C.c_int64)))
    rc = load().mesh_inspect(*args, None, None, None, None)
    if rc != AVIP_OK:
        return rc, None
    E = int(counts[0])
    vol = np.zeros(n)
    edges = np.zeros(2 * max(E, 1), dtype=np.int32)
    S_edge = np.zeros(2 * max(E, 1))
    S_b = np.zeros(2 * n)
    rc = load().mesh_inspect(*args, _dptr(vol), _iptr(edges), _dptr(S_edge), _dptr(S_b))
    return rc, dict(vol=vol, edges=edges[:2 * E].reshape(-1, 2), S_edge=S_edge[:2 * E].reshape(-1, 2),
                    S_b=S_b.reshape(-1, 2), nnz=int(counts[1]), n_cells=int(counts[2]))


def mesh_destroy(h):
    return load().mesh_destroy(h)


def species_set(h, s, charge, mob_model, mob_params, D, bnd_mode, n0):
    mp = np.zeros(4)
    mp[:len(mob_params)] = mob_params
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    return load().species_set(h, s, charge, mob_model, _dptr(mp), float(D), bnd_mode, _dptr(n0))


def source_set(h, model, params, idx):
    p = np.zeros(max(5, len(params)))       # 3 parameters, or 5 for SRC_MORROW_LOWKE
    p[:len(params)] = params
    i = np.ascontiguousarray(idx, dtype=np.int32)
    return load().source_set(h, model, _dptr(p), _iptr(i))


def photo_set(h, a, kappa, c):
    a = np.ascontiguousarray(a, dtype=np.float64)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    return load().photo_set(h, int(a.size), _dptr(a), _dptr(kappa), float(c))


def photo_stats(h):
    """(rc, {"iters": [...], "relres": [...], "side_by_side": bool}) of the last step's
    photoionisation solves."""
    n = C.c_int32(0)
    sbs = C.c_int32(0)
    it = (C.c_int32 * MAX_PHOTO_TERMS)()
    rr = (C.c_double * MAX_PHOTO_TERMS)()
    rc = load().photo_stats(h, C.byref(n), it, rr, C.byref(sbs))
    k = n.value
    return rc, {"iters": list(it)[:k], "relres": list(rr)[:k], "side_by_side": bool(sbs.value)}


def poisson_solve(h):
    it = C.c_int32()
    rr = C.c_double()
    rc = load().poisson_solve(h, C.byref(it), C.byref(rr))
    return rc, it.value, rr.value


def dd_step(h, dt=0.0):
    used = C.c_double()
    rc = load().dd_step(h, float(dt), C.byref(used))
    return rc, used.value


def run_steps(h, nsteps):
    st = AvipStats()
    rc = load().run_steps(h, int(nsteps), C.byref(st))
    return rc, st.as_dict()


TIMED_KERNELS = ("pcg", "node_fields", "dt_cells", "flux_update", "finalize", "photo")


def run_steps_timed(h, nsteps):
    ms = np.zeros(len(TIMED_KERNELS))
    st = AvipStats()
    rc = load().run_steps_timed(h, int(nsteps), _dptr(ms), C.byref(st))
    return rc, dict(zip(TIMED_KERNELS, ms.tolist())), st.as_dict()


def mesh_set_stream(h, stream):
    return load().mesh_set_stream(h, C.c_void_p(stream))


def mesh_set_wait_timeout(h, seconds):
    return load().mesh_set_wait_timeout(h, float(seconds))


def field_get(h, which, s, n_nodes):
    out = np.empty(n_nodes)
    rc = load().field_get(h, which, s, _dptr(out))
    return rc, out


PCG_KINDS = {1: "streaming", 2: "register-resident", 4: "mixed", 5: "cluster-resident", 6: "cluster-mixed",
             7: "bicgstab"}


def mesh_info(h):
    info = np.zeros(8, dtype=np.int64)
    _check(load().mesh_info(h, info.ctypes.data_as(_P(C.c_int64))), "mesh_info")
    return dict(n_nodes=int(info[0]), n_tris=int(info[1]), n_cells=int(info[1]), n_edges=int(info[2]), nnz=int(info[3]),
                pcg_kind=int(info[4]), pcg_blocks=int(info[5]), pcg_threads=int(info[6]),
                device_bytes=int(info[7]))


LEVEL_STATS = 6


def solver_levels(h, max_levels=12):
    """AMG hierarchy of the handle's solver: list of (rows, nnz of A, nnz of P, nnz of Rf,
    nnz of U, nnz of Pf) per level, finest first; empty when the solver is not AMG."""
    out = np.zeros(LEVEL_STATS * max_levels, dtype=np.int64)
    nl = load().solver_levels(h, out.ctypes.data_as(_P(C.c_int64)), max_levels)
    if nl < 0:
        _check(nl, "solver_levels")
    return [tuple(int(v) for v in out[LEVEL_STATS * l:LEVEL_STATS * (l + 1)]) for l in range(min(nl, max_levels))]


def state_get(h, out=None):
    """(rc, state); `out` (float64, contiguous, state_size long, e.g. a view of pinned host
    memory) receives the state when given."""
    n = C.c_int64()
    _check(load().state_size(h, C.byref(n)), "state_size")
    if out is None:
        out = np.empty(n.value)
    elif out.dtype != np.float64 or out.size != n.value or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("state_get: out must be a contiguous float64 array of state_size entries")
    return load().state_get(h, _dptr(out)), out


def state_set(h, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    return load().state_set(h, _dptr(s))


def pcg_csr_static(n, row_ptr, col, val, b, x, rtol, max_iter, stream=0):
    """Jacobi-PCG on a CSR matrix already in device memory, using only the library's
    compiled-in scratch array (no allocation).  Pointer arguments are device addresses (ints,
    e.g. torch tensor .data_ptr()).  Returns (status, iterations, relative residual)."""
    it = C.c_int32()
    rr = C.c_double()
    rc = load().pcg_csr_static(int(n), C.c_void_p(row_ptr), C.c_void_p(col), C.c_void_p(val), C.c_void_p(b),
                               C.c_void_p(x), float(rtol), int(max_iter), C.c_void_p(stream), C.byref(it),
                               C.byref(rr))
    return rc, it.value, rr.value


PROBE_FP64_FMA, PROBE_HBM_COPY = 0, 1


def peak_probe(which, stream=0):
    """Measured FP64 FMA rate (TFLOP/s) or copy bandwidth (GB/s) of the current device."""
    v = C.c_double()
    rc = load().peak_probe(int(which), C.c_void_p(stream), C.byref(v))
    return rc, v.value


def fp64_math_check():
    """Largest relative differences (exp, log, pow, reciprocal) of the library's FP64 math from
    the CUDA math library (the IEEE quotient for the reciprocal)."""
    out = np.zeros(4)
    rc = load().fp64_math_check(_dptr(out))
    return rc, out


def batch_create(handles, cluster_size=0):
    arr = (_H * len(handles))(*[h.value if isinstance(h, _H) else h for h in handles])
    b = _H()
    rc = load().batch_create(arr, len(handles), int(cluster_size), C.byref(b))
    return rc, b


def batch_run_steps(b, nsteps, count):
    st = (AvipStats * count)()
    rc = load().batch_run_steps(b, int(nsteps), C.cast(st, C.c_void_p))
    return rc, [x.as_dict() for x in st]


def batch_info(b):
    info = np.zeros(5, dtype=np.int64)
    _check(load().batch_info(b, info.ctypes.data_as(_P(C.c_int64))), "batch_info")
    return dict(cluster_size=int(info[0]), clusters=int(info[1]), smem_bytes=int(info[2]), count=int(info[3]),
                dd_threads=int(info[4]))


def batch_set_dd_threads(b, threads):
    return load().batch_set_dd_threads(b, int(threads))


def batch_state_get(b, out):
    """Fill `out` (float64, contiguous, the sum of the instances' state sizes) with the batch's
    concatenated states; returns the status."""
    if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("batch_state_get: out must be a contiguous float64 array")
    return load().batch_state_get(b, _dptr(out))


def batch_state_set(b, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    return load().batch_state_set(b, _dptr(s))


def batch_destroy(b):
    return load().batch_destroy(b)


# ------------------------------------------------------------------ convenience wrapper
def torch_allocator():
    """(alloc, free) callbacks drawing device memory from PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    @ALLOC_FN
    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
        except Exception:
            return None

    @FREE_FN
    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return _alloc, _free


class Mesh:
    """Owns one handle built from a synthetic workload (see workloads.Problem)."""

    def __init__(self, problem, precision=PREC_FP64, rtol=None, max_iter=None, dt_fixed=None,
                 reorder=1, use_torch_allocator=False, stream=None, pcg_threads=0, pcg_kind=0,
                 wait_timeout=None, precond_fp64=0, cluster_size=0):
        o = avip_opts_default()
        po = problem.opts
        o.cfl, o.fourier, o.a_diel, o.a_chem = po.cfl, po.fourier, po.a_diel, po.a_chem
        o.beta, o.limiter = po.beta, po.limiter
        o.rtol = po.rtol if rtol is None else rtol
        o.max_iter = po.max_iter if max_iter is None else max_iter
        o.dt_fixed = po.dt_fixed if dt_fixed is None else dt_fixed
        o.precision = precision
        o.reorder = reorder
        o.pcg_threads = pcg_threads
        o.pcg_kind = pcg_kind
        o.geometry = GEOM_AXISYMMETRIC if getattr(problem, "axisymmetric", False) else GEOM_PLANAR
        o.scheme = getattr(po, "scheme", FLUX_LLW)
        o.v_rise = getattr(po, "v_rise", 0.0)
        if wait_timeout is not None:
            o.wait_timeout = wait_timeout
        o.precond_fp64 = int(precond_fp64)
        o.cluster_size = int(cluster_size)
        self._cb = None
        if use_torch_allocator:
            self._cb = torch_allocator()
            o.alloc, o.free = self._cb
        if stream is not None:
            o.stream = C.c_void_p(stream)
        self.problem = problem
        self.N = problem.n_nodes
        quads = getattr(problem, "quads", None)
        if quads is not None and len(quads):
            rc, h = mesh_create_hybrid(problem.xy, problem.tris, quads, problem.node_bc, problem.phi_D, o)
            _check(rc, "mesh_create_hybrid")
        else:
            rc, h = mesh_create(problem.xy, problem.tris, problem.node_bc, problem.phi_D, o)
            _check(rc, "mesh_create")
        self.h = h
        for s, sp in enumerate(problem.species):
            _check(species_set(h, s, sp.charge, sp.mob_model, sp.mob_params, sp.D, sp.bnd_mode, sp.n0),
                   "species_set")
        src = problem.source
        if src.model != 0:
            _check(source_set(h, src.model, src.params, src.idx), "source_set")
        ph = getattr(problem, "photo", None)
        if ph is not None:
            _check(photo_set(h, ph.a, ph.kappa, ph.c), "photo_set")
        self.info = mesh_info(h)
        self.info["levels"] = solver_levels(h)

    def close(self):
        if getattr(self, "h", None):
            mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def poisson_solve(self, allow=(AVIP_OK,)):
        rc, it, rr = poisson_solve(self.h)
        _check(rc, "poisson_solve", allow)
        return it, rr

    def step(self, dt=0.0):
        rc, used = dd_step(self.h, dt)
        _check(rc, "dd_step")
        return used

    def run(self, nsteps, allow=(AVIP_OK,)):
        rc, st = run_steps(self.h, nsteps)
        _check(rc, "run_steps", allow)
        return st

    def run_timed(self, nsteps, allow=(AVIP_OK,)):
        rc, ms, st = run_steps_timed(self.h, nsteps)
        _check(rc, "run_steps_timed", allow)
        return ms, st

    def set_stream(self, stream):
        _check(mesh_set_stream(self.h, stream), "mesh_set_stream")

    def set_wait_timeout(self, seconds):
        _check(mesh_set_wait_timeout(self.h, seconds), "mesh_set_wait_timeout")

    def field(self, which, s=0):
        rc, out = field_get(self.h, which, s, self.N)
        _check(rc, "field_get")
        return out

    def density(self, s):
        return self.field(FIELD_DENSITY, s)

    def phi(self):
        return self.field(FIELD_PHI)

    def photo(self):
        """Photoionisation source S_ph of the last step."""
        return self.field(FIELD_PHOTO)

    def photo_stats(self):
        rc, st = photo_stats(self.h)
        _check(rc, "photo_stats")
        return st

    def state(self, out=None):
        rc, st = state_get(self.h, out)
        _check(rc, "state_get")
        return st

    def set_state(self, st):
        _check(state_set(self.h, st), "state_set")


class Batch:
    """Several Mesh objects advanced together (see batch_create in the C header).  The meshes
    must stay alive, and must not be stepped on their own, while the batch exists."""

    def __init__(self, meshes, cluster_size=0):
        self.meshes = list(meshes)
        rc, b = batch_create([m.h for m in self.meshes], cluster_size)
        _check(rc, "batch_create")
        self.b = b
        self.info = batch_info(b)

    def run(self, nsteps, allow=(AVIP_OK,)):
        rc, st = batch_run_steps(self.b, nsteps, len(self.meshes))
        _check(rc, "batch_run_steps", allow)
        return st

    def state_size(self):
        total = 0
        for m in self.meshes:
            n = C.c_int64()
            _check(load().state_size(m.h, C.byref(n)), "state_size")
            total += n.value
        return total

    def state(self, out=None):
        """The instances' states concatenated (see batch_state_get); `out` may be given."""
        if out is None:
            out = np.empty(self.state_size())
        _check(batch_state_get(self.b, out), "batch_state_get")
        return out

    def set_state(self, st):
        _check(batch_state_set(self.b, st), "batch_state_set")

    def close(self):
        if getattr(self, "b", None):
            batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
