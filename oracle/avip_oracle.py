"""Plain, slow, FP64 CPU oracle for the Poisson-coupled drift-diffusion step of AVIP
(arXiv 2201.01291).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this module;
only the tests, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares
no code with the CUDA library: it restates the paper's vertex-centred finite-volume method
step by step with numpy/scipy, in the paper's order and notation.

Structure (each function cites the passage it follows):
  * metrics: cell volume V_tau, face normals S_f, nodal normals S_k^tau (Eq. node_normal),
    median-dual nodal volume V_i (Fig. 2D_cells), per-cell edge normals S_ij^tau (dual face
    from the edge midpoint to the centroid), boundary nodal normal S_i^b (Fig. bcs_normal);
  * Poisson: matrix of Eq. coeff_matriceA with the sign of the "remark on the implementation"
    (-lap phi = rho/eps0), right-hand side of Eq. poisson_discretization_cartesian, natural
    Neumann rows, Dirichlet values eliminated symmetrically; solved by a sparse direct LU
    (the paper names no linear solver; the exact solution of the linear system is the
    definition being restated);
  * gradients: Green-Gauss cell gradient with nodal normals (section "Cartesian geometry"),
    nodal gradient = volume-weighted mean of the cell gradients (the "centered gradient");
  * transport: limited Lax-Wendroff convective flux with a virtual upwind node and the
    central diffusive flux, accumulated edge by edge (Eq. vertex_centered_flux and the LLW
    section), node-flux boundary closure (section "Boundary conditions in AVIP");
  * time step: cell-based CFL, Fourier, dielectric and chemical limits (section "Time step
    computation");
  * source: ionisation S = alpha mu_e |E| n_e added to electrons and positive ions
    (section "Bagheri benchmark"), optional attachment;
  * Scharfetter-Gummel edge flux as the alternative scheme (section "Scharfetter Gummel
    scheme": exponential fitting on the edge-tangential part of the face normal, centred
    scheme on the normal part);
  * explicit update and the charge sum;
  * axisymmetric (x, r) variant (section "Axisymmetric configuration" and the axisymmetric
    flux form): r-weighted Poisson rows (closed-form dual-contour integral), r-weighted edge
    and boundary normals, dual volumes of revolution; gradients stay two-dimensional;
  * quadrangle and hybrid meshes (n_v-vertex forms of the metrics, section "Nomenclature and
    notations"): shoelace volumes, nodal normals from the two adjacent faces, dual faces from
    the side midpoints to the vertex-mean centre, Poisson coupling of all vertex pairs;
  * three-species air chemistry (section "Hyperbole electrodes": ionisation, attachment,
    electron-ion and ion-ion recombination) and the linear electrode-voltage ramp;
  * photoionisation by the three-term Helmholtz fit (the streamer benchmark's third case):
    (K + kappa_j^2 V) S_j = a_j V I per term, S_ph = sum_j S_j to electrons and positive ions.

Readings where the paper is silent or garbled (each also listed in the design notes):
  * ratio of gradients: r = (u_U - u_k)/(u_W - u_U) with the virtual upwind node
    u_k = u_W - 2 grad(u_U).(x_W - x_U); the printed R_ij is its negative;
  * for V_ij.S_ij < 0 the roles of i and j are mirrored (the 1D form of the limited scheme);
  * u_W == u_U gives Psi = 0;
  * nodal velocity V_s = sign(q_s) mu_s(|E|) E, edge velocity = mean of nodal velocities;
  * Delta x_tau = shortest side of the cell; cell values = mean of the n_v nodal values;
  * chemical time step A_tau * min over nodes of |n_e|/|S_e| (the printed form is not a
    time; the magnitudes keep it a positive time scale when a density undershoots below 0);
  * Dirichlet rows eliminated symmetrically (same solution as the unit-row form);
  * axisymmetric dual volume: the integral of r over the median-dual cell (the centroid
    radius of the dual cell in the Pappus relation; the node radius would give zero volume to
    nodes on the axis); the nodal gradient keeps the planar area weights;
  * node_bc = 2 (a Neumann side's node) is the natural condition, an unknown like 0;
  * photoionisation terms vanish on the Dirichlet nodes and have zero normal derivative on
    the other boundaries; S_ph enters the chemical time-step limit.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12


# ----------------------------------------------------------------------------- metrics
def orient_ccw(xy, tris):
    """Return the triangles with counter-clockwise vertex order (positive signed area)."""
    tris = np.asarray(tris, dtype=np.int64).copy()
    p0, p1, p2 = xy[tris[:, 0]], xy[tris[:, 1]], xy[tris[:, 2]]
    cross = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    flip = cross < 0
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return tris


def cell_volumes(xy, tris):
    """V_tau: area of each (counter-clockwise) triangle."""
    p0, p1, p2 = xy[tris[:, 0]], xy[tris[:, 1]], xy[tris[:, 2]]
    return 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0]))


def face_normals(xy, tris):
    """Outward, length-scaled normals S_f of the three faces of each triangle.
    Face m joins local vertices m and m+1 (mod 3); shape (T, 3, 2)."""
    T = tris.shape[0]
    Sf = np.empty((T, 3, 2))
    for m in range(3):
        p = xy[tris[:, m]]
        q = xy[tris[:, (m + 1) % 3]]
        t = q - p
        Sf[:, m, 0] = t[:, 1]        # right of the direction of travel = outward for CCW
        Sf[:, m, 1] = -t[:, 0]
    return Sf


def nodal_normals(xy, tris):
    """S_k^tau = -(n_d / n_v^f) * sum of the faces adjacent to k (Eq. node_normal);
    triangles: n_d = 2, n_v^f = 2.  Shape (T, 3, 2)."""
    Sf = face_normals(xy, tris)
    S = np.empty_like(Sf)
    for k in range(3):
        # faces adjacent to local vertex k: face k (k -> k+1) and face k-1 (k-1 -> k)
        S[:, k] = -(2.0 / 2.0) * (Sf[:, k] + Sf[:, (k - 1) % 3])
    return S


def nodal_volumes(tris, V_tau, n_nodes):
    """Median-dual nodal volume V_i = sum over E(i) of V_tau / 3 (Fig. 2D_cells)."""
    V = np.zeros(n_nodes)
    for k in range(3):
        np.add.at(V, tris[:, k], V_tau / 3.0)
    return V


def cell_edge_normals(xy, tris):
    """S_ij^tau: length-scaled normal of the dual face inside tau that separates V_i from
    V_j, i.e. the segment from the midpoint of edge (i,j) to the centroid, oriented from i
    towards j (Fig. tri_cell).  Returned for local pairs (0,1), (1,2), (2,0): shape (T,3,2)."""
    c = (xy[tris[:, 0]] + xy[tris[:, 1]] + xy[tris[:, 2]]) / 3.0
    out = np.empty((tris.shape[0], 3, 2))
    for m in range(3):
        xi = xy[tris[:, m]]
        xj = xy[tris[:, (m + 1) % 3]]
        v = c - 0.5 * (xi + xj)
        n = np.stack([v[:, 1], -v[:, 0]], axis=1)
        sgn = np.sign(np.einsum("ij,ij->i", n, xj - xi))
        out[:, m] = n * sgn[:, None]
    return out


def edges_and_normals(xy, tris):
    """Global edge list (i < j) and the aggregated edge normal S_ij = sum_tau S_ij^tau,
    oriented from i to j; also the number of cells sharing each edge."""
    Sc = cell_edge_normals(xy, tris)
    I = np.concatenate([tris[:, m] for m in range(3)])
    J = np.concatenate([tris[:, (m + 1) % 3] for m in range(3)])
    Sv = np.concatenate([Sc[:, m] for m in range(3)])
    swap = I > J
    lo = np.where(swap, J, I)
    hi = np.where(swap, I, J)
    Sv = np.where(swap[:, None], -Sv, Sv)
    key = lo.astype(np.int64) * (int(xy.shape[0]) + 1) + hi
    uniq, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    S = np.zeros((uniq.size, 2))
    np.add.at(S, inv, Sv)
    edges = np.stack([uniq // (int(xy.shape[0]) + 1), uniq % (int(xy.shape[0]) + 1)], axis=1)
    return edges.astype(np.int64), S, counts


def boundary_normals(xy, tris):
    """S_i^b = 1/2 * sum of the outward normals of the boundary faces adjacent to node i
    (Fig. bcs_normal).  A boundary face belongs to exactly one cell."""
    Sf = face_normals(xy, tris)
    I = np.concatenate([tris[:, m] for m in range(3)])
    J = np.concatenate([tris[:, (m + 1) % 3] for m in range(3)])
    F = np.concatenate([Sf[:, m] for m in range(3)])
    lo, hi = np.minimum(I, J), np.maximum(I, J)
    key = lo.astype(np.int64) * (int(xy.shape[0]) + 1) + hi
    _, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    bnd = counts[inv] == 1
    Sb = np.zeros((xy.shape[0], 2))
    np.add.at(Sb, I[bnd], 0.5 * F[bnd])
    np.add.at(Sb, J[bnd], 0.5 * F[bnd])
    return Sb


def min_edge_length(xy, tris):
    """Delta x_tau read as the shortest edge of the cell."""
    L = []
    for m in range(3):
        d = xy[tris[:, (m + 1) % 3]] - xy[tris[:, m]]
        L.append(np.sqrt(d[:, 0] ** 2 + d[:, 1] ** 2))
    return np.minimum(np.minimum(L[0], L[1]), L[2])


# ----------------------------------------------------------------------------- quadrangles
# The same metrics for a group of polygonal cells (C, nv) of one vertex count, used for the
# quadrangles of hybrid meshes (section "Nomenclature and notations": n_v vertices per cell,
# n_v^f = 2 vertices per face, nodal normal S_k = -(n_d/n_v^f) sum of the faces adjacent to k,
# dual volume V_tau/n_v, dual faces from the edge midpoints to the cell centre).
def orient_ccw_poly(xy, cells):
    """Cells with counter-clockwise vertex order (positive shoelace area)."""
    cells = np.asarray(cells, dtype=np.int64).copy()
    flip = poly_volumes(xy, cells) < 0
    cells[flip] = cells[flip, ::-1]
    return cells


def poly_volumes(xy, cells):
    """Signed shoelace area of each polygon."""
    nv = cells.shape[1]
    a = np.zeros(cells.shape[0])
    for m in range(nv):
        p, q = xy[cells[:, m]], xy[cells[:, (m + 1) % nv]]
        a += p[:, 0] * q[:, 1] - q[:, 0] * p[:, 1]
    return 0.5 * a


def poly_face_normals(xy, cells):
    """Outward length-scaled normals of the faces (m, m+1) of counter-clockwise polygons."""
    nv = cells.shape[1]
    Sf = np.empty((cells.shape[0], nv, 2))
    for m in range(nv):
        t = xy[cells[:, (m + 1) % nv]] - xy[cells[:, m]]
        Sf[:, m, 0] = t[:, 1]
        Sf[:, m, 1] = -t[:, 0]
    return Sf


def poly_nodal_normals(xy, cells):
    """S_k = -(n_d / n_v^f) (S_f(k) + S_f(k-1)) with n_d = n_v^f = 2 (Eq. node_normal)."""
    nv = cells.shape[1]
    Sf = poly_face_normals(xy, cells)
    S = np.empty_like(Sf)
    for k in range(nv):
        S[:, k] = -(Sf[:, k] + Sf[:, (k - 1) % nv])
    return S


def poly_edge_normals(xy, cells):
    """Length-scaled normal of the dual face from the midpoint of cell edge (m, m+1) to the
    cell centre (mean of the vertices), oriented from vertex m towards m+1."""
    nv = cells.shape[1]
    c = sum(xy[cells[:, m]] for m in range(nv)) / nv
    out = np.empty((cells.shape[0], nv, 2))
    for m in range(nv):
        xi, xj = xy[cells[:, m]], xy[cells[:, (m + 1) % nv]]
        v = c - 0.5 * (xi + xj)
        n = np.stack([v[:, 1], -v[:, 0]], axis=1)
        sgn = np.sign(np.einsum("ij,ij->i", n, xj - xi))
        out[:, m] = n * sgn[:, None]
    return out


def poly_min_edge_length(xy, cells):
    nv = cells.shape[1]
    L = [np.linalg.norm(xy[cells[:, (m + 1) % nv]] - xy[cells[:, m]], axis=1) for m in range(nv)]
    return np.min(np.stack(L), axis=0)


def poly_poisson_matrix(cells, S, V_tau, n_nodes):
    """K_ik = sum_tau S_i.S_k / (n_d^2 V_tau) over the cells of one group (Eq. coeff_matriceA)."""
    nv = cells.shape[1]
    rows, cols, vals = [], [], []
    for a in range(nv):
        for b in range(nv):
            rows.append(cells[:, a])
            cols.append(cells[:, b])
            vals.append(np.einsum("ij,ij->i", S[:, a], S[:, b]) / (4.0 * V_tau))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n_nodes, n_nodes)).tocsr()


def hybrid_edges_and_boundary(xy, groups):
    """Edge list (i < j) with S_ij summed over every cell of every group, and the boundary
    nodal normals from the faces that belong to one cell only (a face shared by a triangle
    and a quadrangle is interior)."""
    I, J, Sv, F = [], [], [], []
    for cells, Sc, Sf in groups:
        nv = cells.shape[1]
        for m in range(nv):
            I.append(cells[:, m])
            J.append(cells[:, (m + 1) % nv])
            Sv.append(Sc[:, m])
            F.append(Sf[:, m])
    I, J, Sv, F = np.concatenate(I), np.concatenate(J), np.concatenate(Sv), np.concatenate(F)
    n1 = int(xy.shape[0]) + 1
    lo, hi = np.minimum(I, J), np.maximum(I, J)
    Sv = np.where((I > J)[:, None], -Sv, Sv)
    key = lo.astype(np.int64) * n1 + hi
    uniq, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    S = np.zeros((uniq.size, 2))
    np.add.at(S, inv, Sv)
    edges = np.stack([uniq // n1, uniq % n1], axis=1).astype(np.int64)
    bnd = counts[inv] == 1
    Sb = np.zeros((xy.shape[0], 2))
    np.add.at(Sb, I[bnd], 0.5 * F[bnd])
    np.add.at(Sb, J[bnd], 0.5 * F[bnd])
    return edges, S, Sb


# ----------------------------------------------------------------------------- axisymmetry
# Axisymmetric (x, r) configuration: the second coordinate is the radius r >= 0 and every
# volume or face integral carries the weight r (per radian; the common factor 2 pi cancels).
def axi_half_face_integral(xy, tris):
    """Integral of r n dl over the part of the dual contour of vertex k inside each triangle,
    in the closed form of the axisymmetric Poisson section:
      1/24 [(4 r_tau + 2 r_k + r_j + r_l) n_k - (2 r_tau + r_k + r_j) n_j - (2 r_tau + r_k + r_l) n_l]
    with n the nodal normals and r_tau the centroid radius.  Shape (T, 3, 2)."""
    S = nodal_normals(xy, tris)
    r = xy[:, 1][tris]                         # (T, 3)
    rt = r.sum(axis=1) / 3.0
    out = np.empty_like(S)
    for k in range(3):
        j, l = (k + 1) % 3, (k + 2) % 3
        out[:, k] = ((4 * rt + 2 * r[:, k] + r[:, j] + r[:, l])[:, None] * S[:, k]
                     - (2 * rt + r[:, k] + r[:, j])[:, None] * S[:, j]
                     - (2 * rt + r[:, k] + r[:, l])[:, None] * S[:, l]) / 24.0
    return out


def axi_poisson_matrix(xy, tris, V_tau, n_nodes):
    """K_ik = sum_tau (1/(n_d A_tau)) n_k . (integral of r n dl over the dual contour of i in
    tau): the axisymmetric counterpart of Eq. coeff_matriceA for -lap phi = rho/eps0.  Not
    symmetric (the radius breaks the symmetry)."""
    S = nodal_normals(xy, tris)
    I = axi_half_face_integral(xy, tris)
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tris[:, a])
            cols.append(tris[:, b])
            vals.append(np.einsum("ij,ij->i", S[:, b], I[:, a]) / (2.0 * V_tau))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_nodes, n_nodes)).tocsr()
    K.sum_duplicates()
    return K


def axi_nodal_volumes(xy, tris, V_tau):
    """V_i / 2 pi = integral of r over the median-dual cell (second Pappus theorem with the
    centroid radius of the dual cell): per triangle A_tau (22 r_i + 7 r_j + 7 r_k) / 108."""
    r = xy[:, 1][tris]
    V = np.zeros(xy.shape[0])
    for k in range(3):
        j, l = (k + 1) % 3, (k + 2) % 3
        np.add.at(V, tris[:, k], V_tau * (22 * r[:, k] + 7 * r[:, j] + 7 * r[:, l]) / 108.0)
    return V


def axi_edges_and_normals(xy, tris):
    """Edge normals weighted by the radius of their dual face: sum over the cells sharing the
    edge of r_ij^tau S_ij^tau, r_ij^tau the radius at the middle of the dual face (the flux
    form F_ij r_ij^tau S_ij^tau of the axisymmetric flux section)."""
    Sc = cell_edge_normals(xy, tris)
    c = (xy[tris[:, 0], 1] + xy[tris[:, 1], 1] + xy[tris[:, 2], 1]) / 3.0
    I = np.concatenate([tris[:, m] for m in range(3)])
    J = np.concatenate([tris[:, (m + 1) % 3] for m in range(3)])
    rf = np.concatenate([0.5 * (0.5 * (xy[tris[:, m], 1] + xy[tris[:, (m + 1) % 3], 1]) + c) for m in range(3)])
    Sv = np.concatenate([Sc[:, m] for m in range(3)]) * rf[:, None]
    swap = I > J
    lo = np.where(swap, J, I)
    hi = np.where(swap, I, J)
    Sv = np.where(swap[:, None], -Sv, Sv)
    key = lo.astype(np.int64) * (int(xy.shape[0]) + 1) + hi
    uniq, inv = np.unique(key, return_inverse=True)
    S = np.zeros((uniq.size, 2))
    np.add.at(S, inv, Sv)
    edges = np.stack([uniq // (int(xy.shape[0]) + 1), uniq % (int(xy.shape[0]) + 1)], axis=1)
    return edges.astype(np.int64), S


def axi_boundary_normals(xy, tris):
    """Boundary nodal normal weighted by the radius: each boundary face gives its end nodes half
    of its outward normal times the radius at the middle of that half (3 r_p + r_q)/4."""
    Sf = face_normals(xy, tris)
    I = np.concatenate([tris[:, m] for m in range(3)])
    J = np.concatenate([tris[:, (m + 1) % 3] for m in range(3)])
    F = np.concatenate([Sf[:, m] for m in range(3)])
    lo, hi = np.minimum(I, J), np.maximum(I, J)
    key = lo.astype(np.int64) * (int(xy.shape[0]) + 1) + hi
    _, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    bnd = counts[inv] == 1
    rI, rJ = xy[I, 1], xy[J, 1]
    Sb = np.zeros((xy.shape[0], 2))
    np.add.at(Sb, I[bnd], 0.5 * F[bnd] * ((3 * rI[bnd] + rJ[bnd]) / 4.0)[:, None])
    np.add.at(Sb, J[bnd], 0.5 * F[bnd] * ((3 * rJ[bnd] + rI[bnd]) / 4.0)[:, None])
    return Sb


# ----------------------------------------------------------------------------- Poisson
def poisson_matrix(tris, S, V_tau, n_nodes):
    """K = -A with a_ik = sum_tau -S_i.S_k/(V_tau n_d^2) (Eq. coeff_matriceA), i.e. the
    matrix of -lap phi = rho/eps0 (remark on the implementation), n_d = 2."""
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tris[:, a])
            cols.append(tris[:, b])
            vals.append(np.einsum("ij,ij->i", S[:, a], S[:, b]) / (V_tau * 4.0))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_nodes, n_nodes)).tocsr()
    K.sum_duplicates()
    return K


def poisson_rhs(rho, V_node):
    """Right-hand side rho_i V_i / eps0 of Eq. poisson_discretization_cartesian; the zero
    normal field on Neumann sides adds nothing (natural condition)."""
    return rho * V_node / EPS0


class DirichletSolver:
    """Exact solution of K phi = b with phi = phi_D on Dirichlet nodes: the Dirichlet
    columns are moved to the right-hand side and K_FF phi_F = b_F - K_FD phi_D is solved by
    a sparse LU factorisation computed once per mesh."""

    def __init__(self, K, node_bc, phi_D):
        # 1 = Dirichlet; 0 (interior) and 2 (Neumann side: zero normal field, the natural
        # condition of the vertex-centred scheme) are unknowns
        self.free = np.flatnonzero(node_bc != 1)
        self.dir = np.flatnonzero(node_bc == 1)
        self.phi_D = np.asarray(phi_D, dtype=np.float64)
        Kc = K.tocsc()
        self.K_FF = Kc[self.free][:, self.free].tocsc()
        self.K_FD = K.tocsr()[self.free][:, self.dir]
        self.lu = spla.splu(self.K_FF) if self.free.size else None
        self.n = K.shape[0]

    def solve(self, b, gain=1.0):
        """gain scales every Dirichlet value (the voltage ramp of the section "Hyperbole
        electrodes"; 1 for constant electrode potentials)."""
        phi = np.zeros(self.n)
        phi_D = self.phi_D[self.dir] * gain
        phi[self.dir] = phi_D
        if self.free.size:
            rhs = b[self.free] - self.K_FD @ phi_D
            phi[self.free] = self.lu.solve(rhs)
        return phi


# ----------------------------------------------------------------------------- gradients
def cell_gradient(u, tris, S, V_tau):
    """grad u_tau = -1/(V_tau n_d) sum_k u_k S_k (section "Cartesian geometry"), n_d = 2."""
    g = np.zeros((tris.shape[0], 2))
    for k in range(3):
        g += u[tris[:, k]][:, None] * S[:, k]
    return -g / (2.0 * V_tau)[:, None]


def nodal_gradient(u, tris, S, V_tau, V_node):
    """Centered nodal gradient: volume-weighted mean of the cell gradients over E(i), each
    cell contributing its V_tau/3 share of V_i."""
    gc = cell_gradient(u, tris, S, V_tau)
    g = np.zeros((V_node.size, 2))
    for k in range(3):
        np.add.at(g, tris[:, k], gc * (V_tau / 3.0)[:, None])
    return g / V_node[:, None]


# ----------------------------------------------------------------------------- closures
def mobility(sp_, Emag):
    """Mobility of a species as a function of |E|: constant, or the local-field power law
    mu0 (max(|E|, E_floor)/E_ref)^expo."""
    p = sp_.mob_params
    if sp_.mob_model == 0:
        return np.full_like(Emag, p[0])
    if sp_.mob_model == 1:
        return p[0] * (np.maximum(Emag, p[3]) / p[1]) ** p[2]
    raise ValueError("unknown mobility model")


def townsend_alpha(A, B, Emag):
    """alpha(|E|) = A exp(-B/|E|), zero where |E| = 0."""
    out = np.zeros_like(Emag)
    nz = Emag > 0
    out[nz] = A * np.exp(-B / Emag[nz])
    return out


def limiter(r, beta, kind):
    """Psi(r): Sweby(beta) = max(0, min(beta r, 1), min(r, beta)) or Van Leer (r+|r|)/(1+|r|)."""
    if kind == 0:
        return np.maximum(0.0, np.maximum(np.minimum(beta * r, 1.0), np.minimum(r, beta)))
    return (r + np.abs(r)) / (1.0 + np.abs(r))


def bernoulli(x):
    """B(x) = x / (e^x - 1), B(0) = 1 (0 for x beyond the overflow of e^x)."""
    out = np.ones_like(x)
    nz = x != 0
    with np.errstate(over="ignore"):
        out[nz] = x[nz] / np.expm1(x[nz])
    return out


def sg_edge_flux(u_i, u_j, x_i, x_j, S, V, D, g):
    """Scharfetter-Gummel edge flux through the dual face S (oriented i -> j), section
    "Scharfetter Gummel scheme": S is split along the edge direction e = ij/|ij| into
    S_par = (S.e) e and S_perp = S - S_par;
      tangential  V.S_par (u_j - e^a u_i) / (1 - e^a),  a = h V.e / D,  h = |ij|,
      normal      V.S_perp (u_i + u_j)/2 - D g.S_perp   (centred),
    with V the edge velocity and g the mean of the two nodal gradients.  The tangential part
    is evaluated as (D (S.e) / h) (B(-a) u_i - B(a) u_j) with the Bernoulli function B,
    which is the same quantity without the overflow of e^a for |a| > 709 and the 0/0 at a = 0;
    for D = 0 it is the upwind limit (S.e)(max(V.e, 0) u_i + min(V.e, 0) u_j)."""
    d = x_j - x_i
    h = np.sqrt(np.einsum("ij,ij->i", d, d))
    e = d / h[:, None]
    s = np.einsum("ij,ij->i", S, e)
    S_par = s[:, None] * e
    S_perp = S - S_par
    Vt = np.einsum("ij,ij->i", V, e)
    if D > 0:
        a = h * Vt / D
        F_par = (D * s / h) * (bernoulli(-a) * u_i - bernoulli(a) * u_j)
    else:
        F_par = s * (np.maximum(Vt, 0.0) * u_i + np.minimum(Vt, 0.0) * u_j)
    F_perp = np.einsum("ij,ij->i", V, S_perp) * 0.5 * (u_i + u_j) - D * np.einsum("ij,ij->i", g, S_perp)
    return F_par + F_perp


# ----------------------------------------------------------------------------- the method
class Oracle:
    """The full explicit iteration on one mesh.  `problem` is any object with the fields of
    the synthetic workload (xy, tris, node_bc, phi_D, species, source, opts)."""

    def __init__(self, problem):
        self.p = problem
        xy = np.asarray(problem.xy, dtype=np.float64)
        self.xy = xy
        tris = np.asarray(problem.tris, dtype=np.int64).reshape(-1, 3)
        self.tris = orient_ccw(xy, tris) if tris.size else tris
        quads = getattr(problem, "quads", None)
        self.quads = (orient_ccw_poly(xy, np.asarray(quads, dtype=np.int64).reshape(-1, 4))
                      if quads is not None and len(quads) else np.zeros((0, 4), dtype=np.int64))
        self.N = xy.shape[0]
        self.V_tau = cell_volumes(xy, self.tris)
        if np.any(self.V_tau <= 0):
            raise ValueError("degenerate triangle")
        self.V_q = poly_volumes(xy, self.quads)
        if np.any(self.V_q <= 0):
            raise ValueError("degenerate quadrangle")
        self.S_q = poly_nodal_normals(xy, self.quads)
        self.hybrid = self.quads.shape[0] > 0
        self.S = nodal_normals(xy, self.tris)
        # planar dual areas: the weights of the (two-dimensional) nodal gradient
        self.A_node = nodal_volumes(self.tris, self.V_tau, self.N)
        self.dx_tau = min_edge_length(xy, self.tris)
        self.axisymmetric = bool(getattr(problem, "axisymmetric", False))
        if self.hybrid:
            if self.axisymmetric:
                raise ValueError("quadrangles are supported in the planar configuration only")
            for k in range(4):
                np.add.at(self.A_node, self.quads[:, k], self.V_q / 4.0)
            self.dx_q = poly_min_edge_length(xy, self.quads)
            self.V_node = self.A_node
            groups = [(self.quads, poly_edge_normals(xy, self.quads), poly_face_normals(xy, self.quads))]
            if self.tris.size:
                groups.insert(0, (self.tris, cell_edge_normals(xy, self.tris), face_normals(xy, self.tris)))
            self.edges, self.S_edge, self.S_b = hybrid_edges_and_boundary(xy, groups)
            self.K = (poisson_matrix(self.tris, self.S, self.V_tau, self.N)
                      + poly_poisson_matrix(self.quads, self.S_q, self.V_q, self.N)).tocsr()
        elif self.axisymmetric:
            if np.any(xy[:, 1] < 0):
                raise ValueError("axisymmetric meshes need r = y >= 0")
            self.V_node = axi_nodal_volumes(xy, self.tris, self.V_tau)
            self.edges, self.S_edge = axi_edges_and_normals(xy, self.tris)
            self.S_b = axi_boundary_normals(xy, self.tris)
            self.K = axi_poisson_matrix(xy, self.tris, self.V_tau, self.N)
        else:
            self.V_node = self.A_node
            self.edges, self.S_edge, _ = edges_and_normals(xy, self.tris)
            self.S_b = boundary_normals(xy, self.tris)
            self.K = poisson_matrix(self.tris, self.S, self.V_tau, self.N)
        self.node_bc = np.asarray(problem.node_bc)
        self.solver = DirichletSolver(self.K, self.node_bc, problem.phi_D)
        # photoionisation: one Helmholtz operator K + kappa_j^2 V per term, zero on the
        # Dirichlet nodes (the electrodes), zero normal derivative elsewhere
        self.photo = getattr(problem, "photo", None)
        self.photo_solvers = []
        if self.photo is not None:
            for kap in self.photo.kappa:
                H = (self.K + sp.diags(kap * kap * self.V_node)).tocsr()
                self.photo_solvers.append(DirichletSolver(H, self.node_bc, np.zeros(self.N)))
        self.last_photo = np.zeros(self.N)
        self.is_bnd = np.any(self.S_b != 0.0, axis=1)

    # -- Poisson sub-step -------------------------------------------------------------
    def charge_density(self, n):
        rho = np.zeros(self.N)
        for s, sp_ in enumerate(self.p.species):
            rho += E_CHARGE * sp_.charge * n[s]
        return rho

    def dirichlet_gain(self, t):
        """Factor of the electrode potentials at time t: a linear rise from 0 at t = 0 to the
        full value at t = v_rise (Fig. pin-pin_anode_time), then constant; 1 without a ramp."""
        v_rise = getattr(self.p.opts, "v_rise", 0.0)
        if not v_rise > 0:
            return 1.0
        return 1.0 if t >= v_rise else t / v_rise

    def poisson(self, n, t=0.0):
        return self.solver.solve(poisson_rhs(self.charge_density(n), self.V_node), self.dirichlet_gain(t))

    def nodal_gradient(self, u):
        """Centred nodal gradient over all cells (triangles and quadrangles): the cell
        gradients weighted by each cell's V_tau / n_v share of the dual area."""
        if not self.hybrid:
            return nodal_gradient(u, self.tris, self.S, self.V_tau, self.A_node)
        g = np.zeros((self.N, 2))
        for cells, S, V in ((self.tris, self.S, self.V_tau), (self.quads, self.S_q, self.V_q)):
            nv = cells.shape[1]
            if not cells.size:
                continue
            gc = np.zeros((cells.shape[0], 2))
            for k in range(nv):
                gc += u[cells[:, k]][:, None] * S[:, k]
            gc = -gc / (2.0 * V)[:, None]
            for k in range(nv):
                np.add.at(g, cells[:, k], gc * (V / nv)[:, None])
        return g / self.A_node[:, None]

    # -- one explicit step -----------------------------------------------------------
    def fields(self, n, t=0.0):
        """phi, E = -grad phi, |E|, nodal velocities and density gradients at time t."""
        phi = self.poisson(n, t)
        E = -self.nodal_gradient(phi)
        Emag = np.sqrt(E[:, 0] ** 2 + E[:, 1] ** 2)
        mu = [mobility(sp_, Emag) for sp_ in self.p.species]
        vel = [np.sign(sp_.charge) * mu[s][:, None] * E for s, sp_ in enumerate(self.p.species)]
        grad = [self.nodal_gradient(n[s]) for s in range(len(self.p.species))]
        return phi, E, Emag, mu, vel, grad

    def photo_source(self, I):
        """S_ph = sum_j S_j with -lap S_j + kappa_j^2 S_j = a_j I (three-term Helmholtz fit of
        the photoionisation in the streamer benchmark's third case); I is the photon
        production rate c alpha |W_e| n_e.  Integrated over the dual cells:
        (K + kappa_j^2 V) S_j = a_j V I.  Returns S_ph and the terms."""
        terms = [solver.solve(a_j * self.V_node * I) for a_j, solver in zip(self.photo.a, self.photo_solvers)]
        return sum(terms), terms

    def sources(self, n, Emag, mu):
        """Per-species source rates S_s,i (m^-3 s^-1) and the net electron rate."""
        src = self.p.source
        out = [np.zeros(self.N) for _ in self.p.species]
        if src.model == 0:
            return out
        e, pos, neg = src.idx
        A, B = src.params[0], src.params[1]
        nu_att = src.params[2] if src.model == 2 else 0.0
        alpha = townsend_alpha(A, B, Emag)
        ion = alpha * mu[e] * Emag * n[e]
        out[e] = out[e] + ion
        out[pos] = out[pos] + ion
        if src.model == 2:
            att = nu_att * n[e]
            out[e] = out[e] - att
            out[neg] = out[neg] + att
        elif src.model == 3:
            # three-species air chemistry (section "Hyperbole electrodes"): attachment
            # eta |W_e| n_e to the negative ion, electron-ion and ion-ion recombination
            A_eta, B_eta, beta_r = src.params[2], src.params[3], src.params[4]
            att = townsend_alpha(A_eta, B_eta, Emag) * mu[e] * Emag * n[e]
            rec_ep = beta_r * n[e] * n[pos]
            rec_np = beta_r * n[neg] * n[pos]
            out[e] = out[e] - att - rec_ep
            out[pos] = out[pos] - rec_ep - rec_np
            out[neg] = out[neg] + att - rec_np
        if self.photo is not None:
            S_ph, _ = self.photo_source(self.photo.c * ion)
            self.last_photo = S_ph
            out[e] = out[e] + S_ph
            out[pos] = out[pos] + S_ph
        return out

    def time_step(self, n, mu, vel, S_src):
        """Minimum over cells and species of the convective, diffusive and dielectric time
        steps, and the chemical limit over nodes (section "Time step computation")."""
        o = self.p.opts
        dts = [np.inf]
        groups = [(self.tris, self.dx_tau)]
        if self.hybrid:
            groups.append((self.quads, self.dx_q))
        for t, dx in groups:
            if not t.size:
                continue
            nv = t.shape[1]
            for s, sp_ in enumerate(self.p.species):
                Vc = sum(vel[s][t[:, k]] for k in range(nv)) / nv
                Vm = np.sqrt(Vc[:, 0] ** 2 + Vc[:, 1] ** 2)
                ok = Vm > 0
                if np.any(ok):
                    dts.append(np.min(o.cfl * dx[ok] / Vm[ok]))
                if sp_.D > 0:
                    dts.append(np.min(o.fourier * dx ** 2 / sp_.D))
            sigma = np.zeros(t.shape[0])
            for s, sp_ in enumerate(self.p.species):
                nm = n[s] * mu[s]
                cell = sum(nm[t[:, k]] for k in range(nv)) / nv
                sigma += np.abs(sp_.charge * E_CHARGE * cell)
            ok = sigma > 0
            if np.any(ok):
                dts.append(np.min(o.a_diel * EPS0 / sigma[ok]))
        if self.p.source.model != 0:
            e = self.p.source.idx[0]
            Se = S_src[e]
            ok = Se != 0
            if np.any(ok):
                with np.errstate(over="ignore", divide="ignore"):
                    dts.append(np.min(o.a_chem * np.abs(n[e][ok]) / np.abs(Se[ok])))
        return float(min(dts))

    def edge_flux(self, u, grad, vel, D, dt):
        """Limited Lax-Wendroff convective flux plus central diffusive flux through the dual
        face of every edge (i, j), i < j, counted positive from i to j (LLW section and
        "Central difference diffusive flux integration"); or, with opts.scheme = 1, the
        Scharfetter-Gummel flux of sg_edge_flux."""
        o = self.p.opts
        i, j = self.edges[:, 0], self.edges[:, 1]
        S = self.S_edge
        Vij = 0.5 * (vel[i] + vel[j])
        if getattr(o, "scheme", 0) == 1:
            return sg_edge_flux(u[i], u[j], self.xy[i], self.xy[j], S, Vij, D, 0.5 * (grad[i] + grad[j]))
        a = np.einsum("ij,ij->i", Vij, S)
        gij = 0.5 * (grad[i] + grad[j])
        up_i = a >= 0
        U = np.where(up_i, i, j)
        W = np.where(up_i, j, i)
        delta = u[W] - u[U]
        d = self.xy[W] - self.xy[U]
        nz = delta != 0
        r = np.zeros_like(delta)
        r[nz] = (2.0 * np.einsum("ij,ij->i", grad[U][nz], d[nz]) - delta[nz]) / delta[nz]
        psi = np.where(nz, limiter(r, o.beta, o.limiter), 0.0)
        lw = 0.5 * delta - 0.5 * dt * np.einsum("ij,ij->i", gij, Vij)
        FC = (u[U] + lw * psi) * a
        FD = -D * np.einsum("ij,ij->i", gij, S)
        return FC + FD

    def residual(self, u, grad, vel, D, bnd_mode, dt):
        """R_i = -(sum of the fluxes leaving V_i): edge fluxes scattered to both ends
        (Eq. vertex_centered_flux, residual computed at each edge) plus the node-flux
        boundary closure F_i.S_i^b with F = F_C (Neumann) or F_C + F_D (outflow).
        Returns R and the per-node boundary outflow F_i.S_i^b."""
        F = self.edge_flux(u, grad, vel, D, dt)
        R = np.zeros(self.N)
        np.add.at(R, self.edges[:, 0], -F)
        np.add.at(R, self.edges[:, 1], F)
        Fb = u[:, None] * vel
        if bnd_mode == 1:
            Fb = Fb - D * grad
        fb = np.einsum("ij,ij->i", Fb, self.S_b)
        return R - fb, fb

    def step(self, n, dt_fixed=None, t=0.0):
        """One explicit step from densities n (list of (N,) arrays) at time t.  Returns the
        new densities and a dict of diagnostics (phi, E, dt, charge, boundary ledger)."""
        phi, E, Emag, mu, vel, grad = self.fields(n, t)
        S_src = self.sources(n, Emag, mu)
        if dt_fixed is not None and dt_fixed > 0:
            dt = float(dt_fixed)
        elif self.p.opts.dt_fixed > 0:
            dt = float(self.p.opts.dt_fixed)
        else:
            dt = self.time_step(n, mu, vel, S_src)
        new = []
        outflow = []
        for s, sp_ in enumerate(self.p.species):
            R, fb = self.residual(n[s], grad[s], vel[s], sp_.D, sp_.bnd_mode, dt)
            outflow.append(float(np.sum(fb)))
            new.append(n[s] + dt * (R / self.V_node + S_src[s]))
        info = dict(phi=phi, E=E, dt=dt, outflow=outflow,
                    source_total=[float(np.sum(self.V_node * S_src[s])) for s in range(len(n))])
        return new, info

    def charge(self, n):
        """Q = e sum_s q_s sum_i V_i n_s,i."""
        return float(sum(E_CHARGE * sp_.charge * np.sum(self.V_node * n[s])
                         for s, sp_ in enumerate(self.p.species)))

    def initial_state(self):
        return [np.asarray(sp_.n0, dtype=np.float64).copy() for sp_ in self.p.species]

    def run(self, nsteps, n=None):
        """nsteps explicit steps from the initial (or given) state.  Returns the final
        densities, the potential of the last step, and the per-step dt list."""
        n = self.initial_state() if n is None else [x.copy() for x in n]
        dts = []
        phi = None
        t = 0.0
        for _ in range(nsteps):
            n, info = self.step(n, t=t)
            dts.append(info["dt"])
            t = t + info["dt"]
            phi = info["phi"]
        return n, phi, dts
