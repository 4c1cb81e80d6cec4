"""Seeded synthetic inputs for the Poisson-coupled drift-diffusion step.

This module builds *inputs only*: node coordinates, triangles, boundary flags, Dirichlet
values, initial densities and the physical parameters of each species.  It holds none of
the method's arithmetic (no metrics, no fluxes, no solver), so both the CUDA path and the
CPU oracle can be driven from it without sharing any of the method.

Workload shapes follow the drift-diffusion discharge cases of the paper (AVIP, arXiv
2201.01291): a planar domain with two electrodes (Dirichlet potential, Eq. poisson_dirichlet),
insulating sides (zero normal field, Eq. poisson_neumann), electrons and positive ions seeded
by a Gaussian (the initial condition shape of Eq. positive_ions_bagheri, section "Bagheri
benchmark"), on jittered triangle meshes whose sizes span the paper's 1e4--2e6 cells.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

E_CHARGE = 1.602176634e-19      # C
EPS0 = 8.8541878128e-12         # F/m
K_BOLTZMANN = 1.380649e-23      # J/K

# Mobility models understood by both implementations.
MOB_CONST = 0   # mu = mu0
MOB_POWER = 1   # mu = mu0 * (max(|E|, E_floor) / E_ref) ** expo

# Source models.
SRC_NONE = 0
SRC_TOWNSEND = 1            # alpha(|E|) = A exp(-B/|E|);  S = alpha mu_e |E| n_e to e and +
SRC_TOWNSEND_ATTACH = 2     # as above, plus attachment nu_a n_e moved from e to -
SRC_MORROW_LOWKE = 3        # alpha, eta(|E|) attachment, e-p and n-p recombination (params A, B, A_eta, B_eta, beta_r)

# Transport boundary closure modes (section "Boundary conditions in AVIP").
BND_NEUMANN = 0             # F = F_C (zero normal gradient implied)
BND_OUTFLOW = 1             # F = F_C + F_D ("supersonic")

LIM_SWEBY = 0
LIM_VANLEER = 1

FLUX_LLW = 0                # limited Lax-Wendroff convection + central diffusion
FLUX_SG = 1                 # Scharfetter-Gummel on the edge-tangential part, centred normal part


@dataclasses.dataclass
class Species:
    name: str
    charge: int                 # -1 or +1 (units of e)
    mob_model: int
    mob_params: List[float]     # MOB_CONST: [mu0]; MOB_POWER: [mu0, E_ref, expo, E_floor]
    D: float                    # diffusion coefficient, m^2/s
    bnd_mode: int
    n0: np.ndarray              # initial density, m^-3, per node


@dataclasses.dataclass
class Source:
    model: int = SRC_NONE
    params: List[float] = dataclasses.field(default_factory=lambda: [0.0, 0.0, 0.0])  # [A, B, nu_att] or ML's 5
    idx: List[int] = dataclasses.field(default_factory=lambda: [0, 1, -1])  # [electron, positive, negative]


@dataclasses.dataclass
class Photo:
    """Photoionisation by the three-term Helmholtz fit: per term a_j = A_j p_O2^2 (1/m^2) and
    kappa_j = lambda_j p_O2 (1/m); c = (p_q/(p + p_q)) xi nu_u/nu_i scales the ionisation rate."""
    a: List[float]
    kappa: List[float]
    c: float


@dataclasses.dataclass
class Opts:
    cfl: float = 0.4
    fourier: float = 0.25
    a_diel: float = 0.5
    a_chem: float = 0.2
    beta: float = 1.0           # Sweby parameter (1 = min-mod)
    limiter: int = LIM_SWEBY
    rtol: float = 1e-12         # PCG stop: ||b - K phi||_2 <= rtol ||b||_2
    max_iter: int = 20000
    dt_fixed: float = 0.0       # > 0 replaces the automatic time step
    scheme: int = FLUX_LLW      # edge flux scheme
    v_rise: float = 0.0         # > 0: electrode potentials rise linearly over this time (s)


@dataclasses.dataclass
class Problem:
    name: str
    xy: np.ndarray              # (N, 2) float64
    tris: np.ndarray            # (T, 3) int32, counter-clockwise
    node_bc: np.ndarray         # (N,) int32: 0 free, 1 Dirichlet
    phi_D: np.ndarray           # (N,) float64, used where node_bc == 1
    species: List[Species]
    source: Source
    opts: Opts
    seed: int
    meta: dict
    axisymmetric: bool = False   # True: y is the radius r >= 0, x the axis
    quads: Optional[np.ndarray] = None  # (Q, 4) int32 quadrangles of a hybrid mesh
    photo: Optional[Photo] = None       # photoionisation source

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_cells(self) -> int:
        return self.n_tris + (0 if self.quads is None else int(self.quads.shape[0]))


def jittered_rectangle(nx: int, ny: int, Lx: float, Ly: float, jitter: float, seed: int,
                       fixed: Optional[np.ndarray] = None):
    """Structured nx-by-ny node grid on [0,Lx]x[0,Ly], interior nodes moved uniformly in
    +-jitter*h per coordinate, every quad split by its lower-left/upper-right diagonal.
    Nodes are numbered i + nx*j (x fastest).  `fixed` masks extra nodes kept unjittered."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hx, hy = Lx / (nx - 1), Ly / (ny - 1)
    xs = np.arange(nx) * hx
    ys = np.arange(ny) * hy
    X, Y = np.meshgrid(xs, ys)              # (ny, nx)
    X = X.reshape(-1).copy()
    Y = Y.reshape(-1).copy()
    jx = rng.uniform(-jitter * hx, jitter * hx, size=X.shape)
    jy = rng.uniform(-jitter * hy, jitter * hy, size=Y.shape)
    ii = np.tile(np.arange(nx), ny)
    jj = np.repeat(np.arange(ny), nx)
    interior = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < ny - 1)
    if fixed is not None:
        interior &= ~fixed
    X[interior] += jx[interior]
    Y[interior] += jy[interior]
    xy = np.stack([X, Y], axis=1)
    # triangles
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    qi = qi.reshape(-1)
    qj = qj.reshape(-1)
    a = qi + nx * qj
    b = a + 1
    c = a + 1 + nx
    d = a + nx
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    tris = np.empty((2 * a.size, 3), dtype=np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    return xy, tris, ii, jj


def gaussian(xy, x0, y0, sigma, n_peak, n_back):
    r2 = (xy[:, 0] - x0) ** 2 + (xy[:, 1] - y0) ** 2
    return n_peak * np.exp(-r2 / sigma ** 2) + n_back


def default_species(xy, seed_xy, sigma, n_peak, n_back, field_dependent: bool,
                    n_species: int = 2):
    """Electrons + positive ions (+ optional negative ions).  Constant mobility/diffusion
    or the local-field power law mu_e = 0.04 (max(|E|,1e3)/1e6)^-0.2 m^2/Vs."""
    ne = gaussian(xy, seed_xy[0], seed_xy[1], sigma, n_peak, n_back)
    npos = ne.copy()
    if field_dependent:
        e_mob = (MOB_POWER, [0.04, 1e6, -0.2, 1e3])
    else:
        e_mob = (MOB_CONST, [0.04])
    sp = [
        Species("e", -1, e_mob[0], e_mob[1], 0.1, BND_NEUMANN, ne),
        Species("p", +1, MOB_CONST, [2e-4], 5e-6, BND_NEUMANN, npos),
    ]
    if n_species == 3:
        sp.append(Species("n", -1, MOB_CONST, [2.2e-4], 5e-6, BND_NEUMANN,
                          np.full_like(ne, 0.0)))
    return sp


def townsend_air(p_torr: float = 760.0):
    """Textbook air-like Townsend fit alpha = A p exp(-B p/|E|),
    A = 15 /(cm Torr), B = 365 V/(cm Torr), converted to SI."""
    A = 15.0 * 100.0 * p_torr          # 1/m
    B = 365.0 * 100.0 * p_torr         # V/m
    return A, B


def plates_problem(nx: int, ny: int, Lx: float, Ly: float, voltage: float, seed: int,
                   n_peak: float = 1e19, n_back: float = 1e13, sigma: float = 1e-3,
                   jitter: float = 0.2, field_dependent: bool = False, source: int = SRC_NONE,
                   n_species: int = 2, name: str = "plates", opts: Optional[Opts] = None,
                   needle_len: float = 0.0, seed_y: Optional[float] = None) -> Problem:
    """Parallel-plate (optionally pin-plane) discharge: phi = 0 on y = 0, phi = voltage on
    y = Ly (and on a zero-thickness needle of length needle_len hanging from the top centre),
    zero normal field on the sides."""
    fixed = None
    ic = nx // 2
    ii = np.tile(np.arange(nx), ny)
    jj = np.repeat(np.arange(ny), nx)
    hy = Ly / (ny - 1)
    needle = np.zeros(nx * ny, dtype=bool)
    if needle_len > 0:
        needle = (ii == ic) & (jj * hy >= Ly - needle_len - 1e-12 * Ly)
        fixed = needle
    xy, tris, ii, jj = jittered_rectangle(nx, ny, Lx, Ly, jitter, seed, fixed)
    node_bc = np.zeros(nx * ny, dtype=np.int32)
    phi_D = np.zeros(nx * ny, dtype=np.float64)
    bottom = jj == 0
    top = jj == ny - 1
    node_bc[bottom | top | needle] = 1
    phi_D[top | needle] = voltage
    x0 = xy[ic, 0] if needle_len > 0 else 0.5 * Lx
    if seed_y is None:
        seed_y = (Ly - needle_len - 5e-4) if needle_len > 0 else 0.5 * Ly
    sp = default_species(xy, (x0, seed_y), sigma, n_peak, n_back, field_dependent, n_species)
    src = Source()
    if source != SRC_NONE:
        A, B = townsend_air()
        n_gas = 101325.0 / (K_BOLTZMANN * 300.0)
        nu_att = 1e-17 * n_gas if source == SRC_TOWNSEND_ATTACH else 0.0
        src = Source(source, [A, B, nu_att], [0, 1, 2 if n_species == 3 else -1])
    return Problem(name, xy, tris, node_bc, phi_D, sp, src, opts or Opts(), seed,
                   dict(nx=nx, ny=ny, Lx=Lx, Ly=Ly, voltage=voltage, needle_len=needle_len))


def config_small(nx: int = 17, ny: int = 17, seed: int = 7, **kw) -> Problem:
    """Small plates case for fast tests (defaults: 17x17 nodes, 512 triangles)."""
    kw.setdefault("voltage", 5e3)
    return plates_problem(nx, ny, 1e-2, 1e-2, seed=seed, name=f"small{nx}x{ny}", **kw)


def config_plates_65() -> Problem:
    """Plain FP64 parallel plates: 1 cm x 1 cm, 65 x 65 nodes (8192 triangles), jitter +-0.2h,
    seed 1, Gaussian 1e19 m^-3 (sigma 1 mm) at the centre on a 1e13 background, 0 V / 5 kV,
    constant mobility and diffusion, no source, PCG rtol 1e-12, 100 steps."""
    return plates_problem(65, 65, 1e-2, 1e-2, 5e3, seed=1, name="plates65_fp64")


def config_pin_plane(nx: int = 500, ny: int = 1000) -> Problem:
    """Pin-plane streamer: 1 cm x 2 cm, 500 x 1000 nodes (997,002 triangles), 20 kV needle
    anode 2 mm long at the top centre, grounded plane at y = 0, local-field electron mobility
    mu ~ E^-0.2, Townsend ionisation (air-like, 1 atm), Gaussian seed 0.5 mm below the tip."""
    return plates_problem(nx, ny, 1e-2, 2e-2, 2e4, seed=2, field_dependent=True,
                          source=SRC_TOWNSEND, name=f"pin_plane_{nx}x{ny}", needle_len=2e-3)


def config_pin_plane_hybrid(nx: int = 500, ny: int = 1000, quad_fraction: float = 0.5) -> Problem:
    """The pin-plane streamer of config_pin_plane on a hybrid mesh: the same jittered nodes,
    each grid cell kept as a quadrangle with probability quad_fraction, otherwise split into
    two triangles (about 249,500 quadrangles and 499,000 triangles at the default size)."""
    p = hybrid_plates_problem(nx, ny, 1e-2, 2e-2, 2e4, seed=2, quad_fraction=quad_fraction, field_dependent=True,
                              source=SRC_TOWNSEND, needle_len=2e-3)
    return dataclasses.replace(p, name=f"pin_plane_hybrid_{nx}x{ny}_q{quad_fraction:g}")


def morrow_lowke_air(T_gas: float = 1000.0, p_atm: float = 1.0):
    """Analytic closure fits for the three-species air chemistry at gas temperature T_gas
    (project choices standing in for the tabulated coefficients, which are not available): the
    reduced-field similarity of the Townsend fit with the density-equivalent pressure
    p = 760 p_atm (300 / T_gas) Torr; attachment eta = 1.3 p /(m Torr) exp(-B_eta/|E|) with
    B_eta = 20 p V/(m Torr) (about 10 /cm at breakdown at 1 atm, 300 K); recombination
    beta_r = 2e-13 m^3/s; electron mobility mu_e = (T_gas/300) 0.04 (max(|E|, 1e3)/E_ref)^-0.2
    with E_ref = 1e6 (300 / T_gas) V/m.  Returns (source params, electron mobility params)."""
    p_torr = 760.0 * p_atm * 300.0 / T_gas
    A, B = townsend_air(p_torr)
    A_eta, B_eta = 1.3 * p_torr, 20.0 * p_torr
    beta_r = 2e-13
    s = T_gas / 300.0
    mob = [0.04 * s / p_atm, 1e6 / s * p_atm, -0.2, 1e3]
    return [A, B, A_eta, B_eta, beta_r], mob


def morrow_lowke_problem(nx: int, ny: int, Lx: float, Ly: float, v_max: float, seed: int,
                         needle_len: float = 0.0, T_gas: float = 1000.0, v_rise: float = 2e-9,
                         n_back: float = 1e15, quad_fraction: float = 0.0, **kw) -> Problem:
    """Three-species (e, p, n) air chemistry of the section "Hyperbole electrodes" on the
    pin-plane geometry: immobile ions (the ion equations carry no transport term), a uniform
    neutral background of electrons and positive ions, and the anode potential rising linearly
    from 0 to v_max over v_rise (Fig. pin-pin_anode_time).  quad_fraction > 0 builds a hybrid
    mesh."""
    if quad_fraction > 0:
        p = hybrid_plates_problem(nx, ny, Lx, Ly, v_max, seed, quad_fraction=quad_fraction, n_peak=0.0,
                                  n_back=n_back, needle_len=needle_len, **kw)
    else:
        p = plates_problem(nx, ny, Lx, Ly, v_max, seed, n_peak=0.0, n_back=n_back, needle_len=needle_len, **kw)
    params, mob = morrow_lowke_air(T_gas)
    N = p.n_nodes
    sp = [
        Species("e", -1, MOB_POWER, mob, 0.1 * T_gas / 300.0, BND_OUTFLOW, np.full(N, n_back)),
        Species("p", +1, MOB_CONST, [0.0], 0.0, BND_NEUMANN, np.full(N, n_back)),
        Species("n", -1, MOB_CONST, [0.0], 0.0, BND_NEUMANN, np.zeros(N)),
    ]
    opts = dataclasses.replace(p.opts, v_rise=v_rise)
    return dataclasses.replace(p, species=sp, source=Source(SRC_MORROW_LOWKE, params, [0, 1, 2]), opts=opts,
                               name=f"morrow_lowke_{nx}x{ny}")


def config_hyperbole_ml(nx: int = 800, ny: int = 800) -> Problem:
    """Stand-in for the hyperbolic-electrode case: a 5 mm x 5 mm gap, 1 mm needle anode at the
    top centre rising to 5 kV in 2 ns, grounded plane, 1000 K air (three-species chemistry),
    1e15 m^-3 background; 800 x 800 jittered nodes (640,000 nodes, 1.28 M triangles, the size of
    the paper's 6.3e5-node, 1.3e6-cell mesh)."""
    return morrow_lowke_problem(nx, ny, 5e-3, 5e-3, 5e3, seed=1745, needle_len=1e-3)


def photo_air(p_torr: float = 760.0, p_q_torr: float = 30.0, xi_ratio: float = 0.06) -> Photo:
    """Three-term fit for air: A_j = (1.986e-4, 0.0051, 0.4886) /(cm^2 Torr^2) and lambda_j =
    (0.0553, 0.146, 0.89) /(cm Torr), p_O2 = 0.2 p, quenching pressure p_q = 30 Torr and
    xi nu_u/nu_i = 0.06 (inputs of this stand-in: the values commonly quoted for the fit, not
    checked here against the original tables)."""
    p_o2 = 0.2 * p_torr
    A = [1.986e-4, 0.0051, 0.4886]
    lam = [0.0553, 0.146, 0.89]
    a = [Aj * p_o2 ** 2 * 1e4 for Aj in A]
    kappa = [lj * p_o2 * 1e2 for lj in lam]
    return Photo(a, kappa, p_q_torr / (p_torr + p_q_torr) * xi_ratio)


def config_axisym_photo(nx: int = 701, ny: int = 701) -> Problem:
    """The axisymmetric streamer gap of config_axisym_streamer with a 1e9 m^-3 background and
    photoionisation (the benchmark's third case: its second case plus photoionisation)."""
    p = config_axisym_streamer(nx, ny, n_back=1e9)
    return dataclasses.replace(p, photo=photo_air(), name=f"axisym_photo_{nx}x{ny}")


def random_instances(count: int, seed: int, t_min: float = 2e3, t_max: float = 2e5):
    """Many uneven discharge instances: triangle counts log-uniform in [t_min, t_max], aspect
    ratio uniform in [1,4], voltage uniform in [5,25] kV, 2 or 3 charged species (the third a
    negative ion fed by attachment, k = 1e-17 m^3/s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        T = float(np.exp(rng.uniform(np.log(t_min), np.log(t_max))))
        ar = float(rng.uniform(1.0, 4.0))
        volt = float(rng.uniform(5e3, 25e3))
        ns = int(rng.integers(2, 4))
        # T = 2 (nx-1)(ny-1), ny-1 = ar (nx-1)
        nq = max(1.0, np.sqrt(T / (2.0 * ar)))
        nx = max(5, int(round(nq)) + 1)
        ny = max(5, int(round(nq * ar)) + 1)
        Lx = 1e-2
        Ly = Lx * (ny - 1) / (nx - 1)
        src = SRC_TOWNSEND_ATTACH if ns == 3 else SRC_TOWNSEND
        p = plates_problem(nx, ny, Lx, Ly, volt, seed=seed * 100003 + k, field_dependent=True,
                           source=src, n_species=ns, name=f"inst{k}")
        out.append(p)
    return out


def axisym_problem(nx: int, nr: int, Lx: float, Lr: float, voltage: float, seed: int,
                   n_peak: float = 1e19, n_back: float = 1e13, sigma: float = 1e-3, jitter: float = 0.2,
                   field_dependent: bool = False, source: int = SRC_NONE, n_species: int = 2,
                   x0: Optional[float] = None, name: str = "axisym", opts: Optional[Opts] = None) -> Problem:
    """Axisymmetric (x, r) plane-to-plane gap: x is the axis, y = r the radius (the axis y = 0
    and the outer radius carry no condition: zero normal field), phi = 0 on x = 0 and
    phi = voltage on x = Lx; Gaussian seed on the axis at x0 (default mid-gap)."""
    xy, tris, ii, jj = jittered_rectangle(nx, nr, Lx, Lr, jitter, seed)
    node_bc = np.zeros(nx * nr, dtype=np.int32)
    phi_D = np.zeros(nx * nr, dtype=np.float64)
    left = ii == 0
    right = ii == nx - 1
    node_bc[left | right] = 1
    phi_D[right] = voltage
    x0 = 0.5 * Lx if x0 is None else x0
    sp = default_species(xy, (x0, 0.0), sigma, n_peak, n_back, field_dependent, n_species)
    src = Source()
    if source != SRC_NONE:
        A, B = townsend_air()
        n_gas = 101325.0 / (K_BOLTZMANN * 300.0)
        nu_att = 1e-17 * n_gas if source == SRC_TOWNSEND_ATTACH else 0.0
        src = Source(source, [A, B, nu_att], [0, 1, 2 if n_species == 3 else -1])
    return Problem(name, xy, tris, node_bc, phi_D, sp, src, opts or Opts(), seed,
                   dict(nx=nx, nr=nr, Lx=Lx, Lr=Lr, voltage=voltage), axisymmetric=True)


def config_axisym_streamer(nx: int = 701, nr: int = 701, seed: int = 2201, n_back: float = 1e13) -> Problem:
    """Axisymmetric streamer gap in the geometry of the paper's axisymmetric streamer benchmark
    (section "Bagheri benchmark"): 1.25 cm x 1.25 cm, 1.5 MV/m background field (18.75 kV),
    Gaussian seed of 5e18 m^-3 (sigma 0.4 mm) on the axis at x = 1 cm over a 1e13 m^-3
    background; local-field electron mobility and Townsend ionisation of this library's models
    (the benchmark's tabulated transport data are not used).  701 x 701 nodes: 980,000
    triangles, the size class of the pin-plane workload."""
    return axisym_problem(nx, nr, 1.25e-2, 1.25e-2, 18750.0, seed, n_peak=5e18, n_back=n_back, sigma=4e-4,
                          field_dependent=True, source=SRC_TOWNSEND, x0=1e-2, name="axisym_streamer")


def hybrid_plates_problem(nx: int, ny: int, Lx: float, Ly: float, voltage: float, seed: int,
                          quad_fraction: float = 1.0, **kw) -> Problem:
    """The parallel-plate problem of plates_problem on a quadrangle or hybrid mesh: the same
    jittered node grid, each grid cell kept as a quadrangle with probability quad_fraction
    (seeded), otherwise split into two triangles along its lower-left/upper-right diagonal."""
    p = plates_problem(nx, ny, Lx, Ly, voltage, seed, **kw)
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    a = (qi + nx * qj).reshape(-1)
    b, c, d = a + 1, a + 1 + nx, a + nx
    rng = np.random.Generator(np.random.PCG64(seed + 7777))
    keep = rng.uniform(size=a.size) < quad_fraction
    quads = np.stack([a, b, c, d], axis=1)[keep].astype(np.int32)
    t1 = np.stack([a, b, c], axis=1)[~keep]
    t2 = np.stack([a, c, d], axis=1)[~keep]
    tris = np.concatenate([t1, t2]).astype(np.int32).reshape(-1, 3)
    return dataclasses.replace(p, tris=tris, quads=quads, name=f"hybrid_{nx}x{ny}_q{quad_fraction:g}")
