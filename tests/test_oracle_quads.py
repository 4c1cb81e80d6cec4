"""Pins of the oracle on quadrangle and hybrid (triangle + quadrangle) meshes: polygon metrics
(nodal normals sum to zero, areas, dual areas tile the domain, closure of the dual contours),
Green-Gauss gradients exact on linear fields, the Poisson operator annihilating linear fields
at interior rows and converging at second order on a manufactured solution, the linear
potential between plates, the one-dimensional limited Lax-Wendroff scheme on an unjittered
quadrangle strip (and the one-dimensional Scharfetter-Gummel scheme), a uniform state preserved
and the charge ledger.  CPU only."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


def hybrid(nx=11, ny=9, frac=0.5, seed=3, **kw):
    return W.hybrid_plates_problem(nx, ny, 1e-2, 0.8e-2, 5e3, seed=seed, quad_fraction=frac, **kw)


def test_polygon_metrics():
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [2.5, 1.0], [0.2, 1.5]])
    q = np.array([[0, 3, 2, 1]])                       # clockwise on input
    q = O.orient_ccw_poly(xy, q)
    assert O.poly_volumes(xy, q)[0] > 0
    # shoelace area of the quadrangle by triangle fan
    cross = lambda a, b: a[0] * b[1] - a[1] * b[0]
    fan = 0.5 * abs(cross(xy[1] - xy[0], xy[2] - xy[0])) + 0.5 * abs(cross(xy[2] - xy[0], xy[3] - xy[0]))
    assert abs(O.poly_volumes(xy, q)[0] - fan) < 1e-15
    S = O.poly_nodal_normals(xy, q)
    assert np.abs(S.sum(axis=1)).max() < 1e-15
    # Green-Gauss: -1/(2V) sum u_k S_k is exact for a linear u
    u = 0.3 - 1.7 * xy[:, 0] + 2.2 * xy[:, 1]
    g = -(u[q[0]][:, None] * S[0]).sum(axis=0) / (2.0 * O.poly_volumes(xy, q)[0])
    np.testing.assert_allclose(g, [-1.7, 2.2], rtol=1e-14)
    # the dual faces of each vertex close its part of the cell: sum over the two faces of the
    # vertex of the dual normals equals S_k / n_d
    Sc = O.poly_edge_normals(xy, q)[0]
    for k in range(4):
        np.testing.assert_allclose(Sc[k] - Sc[(k - 1) % 4], S[0, k] / 2.0, atol=1e-15)


@pytest.mark.parametrize("frac", [1.0, 0.5])
def test_hybrid_closure_areas_and_gradient(frac):
    p = hybrid(frac=frac)
    o = O.Oracle(p)
    assert o.hybrid
    assert abs(o.A_node.sum() - 1e-2 * 0.8e-2) < 1e-18
    # closure: sum of the edge normals leaving a node plus its boundary normal is zero
    C = np.zeros((o.N, 2))
    np.add.at(C, o.edges[:, 0], o.S_edge)
    np.add.at(C, o.edges[:, 1], -o.S_edge)
    C += o.S_b
    assert np.abs(C).max() < 1e-18
    u = 1.0 + 300.0 * p.xy[:, 0] - 700.0 * p.xy[:, 1]
    np.testing.assert_allclose(o.nodal_gradient(u), np.tile([300.0, -700.0], (o.N, 1)), rtol=1e-11)
    # the operator annihilates linear fields at interior rows and constants everywhere
    nx, ny = 11, 9
    ii, jj = np.tile(np.arange(nx), ny), np.repeat(np.arange(ny), nx)
    interior = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < ny - 1)
    assert np.abs((o.K @ u)[interior]).max() < 1e-9 * np.abs(o.K).max() * np.abs(u).max()
    assert np.abs(o.K @ np.ones(o.N)).max() < 1e-12 * np.abs(o.K).max()


def test_quadrangle_manufactured_second_order():
    """phi = x^2 + y^2 (-lap phi = -4) with Dirichlet data on the whole boundary of the unit
    square, on jittered quadrangle meshes."""
    errs = []
    for n in (9, 17, 33, 65):
        p = W.hybrid_plates_problem(n, n, 1.0, 1.0, 0.0, seed=5, quad_fraction=1.0, n_peak=0.0, n_back=0.0)
        xy = p.xy
        ii, jj = np.tile(np.arange(n), n), np.repeat(np.arange(n), n)
        bc = ((ii == 0) | (ii == n - 1) | (jj == 0) | (jj == n - 1)).astype(np.int32)
        q = O.orient_ccw_poly(xy, p.quads)
        V = O.poly_volumes(xy, q)
        K = O.poly_poisson_matrix(q, O.poly_nodal_normals(xy, q), V, n * n)
        Vn = np.zeros(n * n)
        for k in range(4):
            np.add.at(Vn, q[:, k], V / 4.0)
        f = xy[:, 0] ** 2 + xy[:, 1] ** 2
        phi = O.DirichletSolver(K, bc, f).solve(O.poisson_rhs(np.full(n * n, -4.0 * O.EPS0), Vn))
        errs.append(np.abs(phi - f).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3 and rates[1:].mean() > 1.6, (errs, rates)


def test_hybrid_plates_linear_potential_exact():
    p = hybrid(13, 11, 0.5, n_peak=0.0, n_back=0.0)
    o = O.Oracle(p)
    phi = o.poisson(o.initial_state())
    np.testing.assert_allclose(phi, 5e3 * p.xy[:, 1] / 0.8e-2, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("c", [3.0, -2.0])
def test_quad_strip_reduces_to_1d_limited_lax_wendroff(c):
    """On an unjittered quadrangle strip with u = u(x), V = (c, 0), the 2D residual per unit
    face height equals the textbook 1D limited Lax-Wendroff residual with real upwind nodes and
    centred nodal gradients (the virtual upwind node coincides with the grid node)."""
    nx, ny = 24, 8
    h = 1.0 / (nx - 1)
    p = W.hybrid_plates_problem(nx, ny, 1.0, h * (ny - 1), 0.0, seed=1, quad_fraction=1.0, jitter=0.0,
                                n_peak=0.0, n_back=0.0)
    o = O.Oracle(p)
    prof = lambda xx: 1e2 + 0.5 * (1.0 + np.tanh((xx - 0.45) / 0.08)) * 1e6 + 3e5 * np.sin(7 * xx)
    u = prof(p.xy[:, 0])
    grad = o.nodal_gradient(u)
    vel = np.tile([c, 0.0], (p.n_nodes, 1))
    dt, D = 0.01, 0.05
    R, _ = o.residual(u, grad, vel, D, 0, dt)
    U = prof(np.arange(nx) * h)
    g = np.zeros(nx)
    g[1:-1] = (U[2:] - U[:-2]) / (2 * h)

    def face(i):
        up, dn, uu = (i, i + 1, i - 1) if c >= 0 else (i + 1, i, i + 2)
        delta = U[dn] - U[up]
        psi = 0.0
        if delta != 0:
            r = (U[up] - U[uu]) / delta
            psi = max(0.0, min(r, 1.0), min(r, 1.0))
        gf = 0.5 * (g[i] + g[i + 1])
        return (U[up] + (0.5 * delta - 0.5 * dt * gf * c) * psi) * c - D * gf

    ii, jj = np.tile(np.arange(nx), ny), np.repeat(np.arange(ny), nx)
    sel = (ii >= 3) & (ii <= nx - 4) & (jj >= 2) & (jj <= ny - 3)
    R1 = np.array([-(face(i) - face(i - 1)) for i in ii[sel]])
    np.testing.assert_allclose(R[sel] / h, R1, atol=1e-12 * np.abs(U).max() * abs(c))


def test_hybrid_uniform_state_and_charge_ledger():
    q = hybrid(13, 11, 0.5, n_peak=0.0, n_back=1e12)
    oq = O.Oracle(q)
    m = oq.initial_state()
    for _ in range(3):
        m, _ = oq.step(m)
    for s in range(2):
        np.testing.assert_allclose(m[s], 1e12, rtol=1e-12)
    p = W.hybrid_plates_problem(17, 15, 1e-2, 1e-2, 2e4, seed=4, quad_fraction=0.6, field_dependent=True,
                                source=W.SRC_TOWNSEND)
    o = O.Oracle(p)
    n = o.initial_state()
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n)
    for _ in range(6):
        Q0 = o.charge(n)
        n, info = o.step(n)
        ledger = sum(-info["dt"] * O.E_CHARGE * sp_.charge * (info["outflow"][s] - info["source_total"][s])
                     for s, sp_ in enumerate(p.species))
        assert abs(o.charge(n) - Q0 - ledger) <= 1e-13 * scale


@pytest.mark.parametrize("c", [3.0, -2.0])
def test_quad_strip_reduces_to_1d_scharfetter_gummel(c):
    """On an unjittered quadrangle strip the dual faces are normal to the edges (no normal part
    of S): with u = u(x) and V = (c, 0) the residual per unit face height is the textbook 1D
    Scharfetter-Gummel one, F_{i+1/2} = (D/h) (B(-a) u_i - B(a) u_{i+1}), a = h c / D."""
    nx, ny = 24, 8
    h = 1.0 / (nx - 1)
    p = W.hybrid_plates_problem(nx, ny, 1.0, h * (ny - 1), 0.0, seed=1, quad_fraction=1.0, jitter=0.0,
                                n_peak=0.0, n_back=0.0)
    p.opts.scheme = W.FLUX_SG
    o = O.Oracle(p)
    prof = lambda xx: 1e2 + 0.5 * (1.0 + np.tanh((xx - 0.45) / 0.08)) * 1e6 + 3e5 * np.sin(7 * xx)
    u = prof(p.xy[:, 0])
    vel = np.tile([c, 0.0], (p.n_nodes, 1))
    D = 0.05
    R, _ = o.residual(u, o.nodal_gradient(u), vel, D, 0, 0.01)
    U = prof(np.arange(nx) * h)
    a = h * c / D
    B = lambda x: x / np.expm1(x)
    face = lambda i: (D / h) * (B(-a) * U[i] - B(a) * U[i + 1])
    ii, jj = np.tile(np.arange(nx), ny), np.repeat(np.arange(ny), nx)
    sel = (ii >= 1) & (ii <= nx - 2) & (jj >= 1) & (jj <= ny - 2)
    R1 = np.array([-(face(i) - face(i - 1)) for i in ii[sel]])
    np.testing.assert_allclose(R[sel] / h, R1, rtol=0, atol=1e-11 * np.abs(U).max() * (abs(c) + D / h))
