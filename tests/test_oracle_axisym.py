"""Pins of the oracle's axisymmetric (x, r) variant: the closed-form dual-contour integral of
the axisymmetric Poisson section against Gauss quadrature, exact volumes of revolution, exact
action of the operator on linear fields, second-order convergence of a manufactured
solution, the planar limit far from the axis, charge conservation and preservation of a
uniform state in an axial field.  CPU only."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


def mesh(nx=9, nr=7, Lx=1.0, Lr=0.8, r0=0.0, seed=3):
    xy, tris, ii, jj = W.jittered_rectangle(nx, nr, Lx, Lr, 0.2, seed)
    xy = xy.copy()
    xy[:, 1] += r0
    return xy, O.orient_ccw(xy, tris), ii, jj


def test_half_face_integral_matches_quadrature():
    """Closed form == 3-point Gauss quadrature of r n dl along the two dual segments
    (edge midpoint -> centroid) of each vertex, normals pointing out of the vertex's cell."""
    xy, t, _, _ = mesh()
    I = O.axi_half_face_integral(xy, t)
    g = np.array([0.5 - np.sqrt(15) / 10, 0.5, 0.5 + np.sqrt(15) / 10])
    w = np.array([5, 8, 5]) / 18.0
    for c in range(t.shape[0]):
        P = xy[t[c]]
        cen = P.mean(axis=0)
        for k in range(3):
            acc = np.zeros(2)
            for j in ((k + 1) % 3, (k + 2) % 3):
                m = 0.5 * (P[k] + P[j])
                seg = cen - m
                nrm = np.array([seg[1], -seg[0]])
                if nrm @ (P[j] - P[k]) < 0:
                    nrm = -nrm          # away from vertex k
                rq = (m + np.outer(g, seg))[:, 1]
                acc += nrm * (w @ rq)
            np.testing.assert_allclose(I[c, k], acc, rtol=1e-12, atol=1e-15)


def test_volumes_of_revolution_exact():
    for r0 in (0.0, 0.3):
        xy, t, _, _ = mesh(nx=11, nr=6, Lx=2.0, Lr=0.5, r0=r0)
        V = O.axi_nodal_volumes(xy, t, O.cell_volumes(xy, t))
        exact = 2.0 * ((r0 + 0.5) ** 2 - r0 ** 2) / 2.0      # integral of r over the rectangle
        assert abs(V.sum() - exact) < 1e-13
        assert np.all(V > 0)                                  # also on the axis


def test_operator_on_linear_fields():
    """K x = 0 and (K r)_i = -A_i (planar dual area) at interior nodes: the dual-contour
    integrals are exact for fields linear in x and r."""
    nx, nr = 10, 9
    xy, t, ii, jj = mesh(nx=nx, nr=nr)
    V = O.cell_volumes(xy, t)
    K = O.axi_poisson_matrix(xy, t, V, xy.shape[0])
    A = O.nodal_volumes(t, V, xy.shape[0])
    interior = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < nr - 1)
    assert np.abs((K @ xy[:, 0])[interior]).max() < 1e-12
    np.testing.assert_allclose((K @ xy[:, 1])[interior], -A[interior], rtol=1e-11)
    assert np.abs(K - K.T).max() > 1e-6                       # the radius breaks the symmetry


def test_manufactured_axisymmetric_second_order():
    """phi = x^2 + r^2: lap_axi phi = 2 + 2 + 2 = 6, i.e. rho/eps0 = -6; Dirichlet on x = 0,
    x = 1 and r = 1, nothing on the axis (the solution has zero radial slope there)."""
    errs = []
    for n in (9, 17, 33):
        xy, t, ii, jj = W.jittered_rectangle(n, n, 1.0, 1.0, 0.2, 21)
        t = O.orient_ccw(xy, t)
        V = O.cell_volumes(xy, t)
        K = O.axi_poisson_matrix(xy, t, V, xy.shape[0])
        Vn = O.axi_nodal_volumes(xy, t, V)
        bc = ((ii == 0) | (ii == n - 1) | (jj == n - 1)).astype(np.int32)
        f = xy[:, 0] ** 2 + xy[:, 1] ** 2
        phi = O.DirichletSolver(K, bc, f).solve(O.poisson_rhs(np.full(xy.shape[0], -6.0 * O.EPS0), Vn))
        errs.append(np.abs(phi - f).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3 and rates.mean() > 1.5, (errs, rates)


def test_planar_limit_far_from_axis():
    r0 = 1e4
    xy, t, _, _ = mesh(r0=r0)
    V = O.cell_volumes(xy, t)
    Ka = O.axi_poisson_matrix(xy, t, V, xy.shape[0]).toarray() / r0
    xy0 = xy.copy()
    xy0[:, 1] -= r0
    Kp = O.poisson_matrix(t, O.nodal_normals(xy0, t), O.cell_volumes(xy0, t), xy.shape[0]).toarray()
    assert np.abs(Ka - Kp).max() <= 1e-3 * np.abs(Kp).max()


def test_axisymmetric_charge_ledger_and_axial_uniform_state():
    p = W.axisym_problem(17, 13, 1e-2, 0.6e-2, 2e4, seed=4, source=W.SRC_TOWNSEND, field_dependent=True)
    o = O.Oracle(p)
    n = o.initial_state()
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n)
    for _ in range(8):
        Q0 = o.charge(n)
        n, info = o.step(n)
        ledger = sum(-info["dt"] * O.E_CHARGE * sp_.charge * (info["outflow"][s] - info["source_total"][s])
                     for s, sp_ in enumerate(p.species))
        assert abs(o.charge(n) - Q0 - ledger) <= 1e-13 * scale
    # neutral uniform plasma in the axial field of the plates: transport leaves it unchanged
    q = W.axisym_problem(13, 11, 1e-2, 0.5e-2, 5e3, seed=6, n_peak=0.0, n_back=1e12)
    oq = O.Oracle(q)
    m = oq.initial_state()
    for _ in range(3):
        m, _ = oq.step(m)
    for s in range(2):
        np.testing.assert_allclose(m[s], 1e12, rtol=1e-12)
