"""Pins of the oracle's Scharfetter-Gummel edge flux (section "Scharfetter Gummel scheme"):
exactness on the exponential steady profile of drift-diffusion along the edge, the centred
normal part, the upwind and pure-diffusion limits, antisymmetry, and conservation properties
of a whole step with the scheme.  CPU only."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


def one_edge(theta, h, s_par, s_perp):
    e = np.array([np.cos(theta), np.sin(theta)])
    n = np.array([-e[1], e[0]])
    x_i = np.array([[0.3, -0.2]])
    x_j = x_i + h * e
    S = (s_par * e + s_perp * n)[None, :]
    return x_i, x_j, e, n, S


@pytest.mark.parametrize("alpha", [-800.0, -35.0, -2.0, -1e-3, 1e-9, 0.7, 12.0, 400.0])
def test_exact_on_exponential_steady_profile(alpha):
    """u(xi) = A + B exp(V xi / D) carries the constant flux V u - D u' = V A along the edge;
    the tangential SG flux reproduces it exactly for any cell Peclet number a = h V / D."""
    h, D, A = 2e-5, 0.1, 3.0e15
    Vt = alpha * D / h
    B = 1e14 * np.exp(-max(alpha, 0.0))          # keep u_j finite for large positive a
    theta = 0.37
    x_i, x_j, e, n, S = one_edge(theta, h, 1.7e-5, 0.0)
    u_i = np.array([A + B])
    u_j = np.array([A + B * np.exp(alpha)])
    V = (Vt * e)[None, :]
    F = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, V, D, np.zeros((1, 2)))
    exact = Vt * A * 1.7e-5
    scale = abs(Vt) * (abs(A) + abs(B) + B * np.exp(alpha)) * 1.7e-5
    assert abs(F[0] - exact) <= 1e-12 * scale


def axis_edge(h, s_par, s_perp):
    """Edge along +y with binary-exact end points, so e = (0, 1) and S.e are exact."""
    x_i = np.array([[0.25, -0.125]])
    x_j = x_i + np.array([[0.0, h]])
    e, n = np.array([0.0, 1.0]), np.array([-1.0, 0.0])
    return x_i, x_j, e, n, (s_par * e + s_perp * n)[None, :]


def test_normal_part_is_centred():
    """S perpendicular to the edge: V.S (u_i + u_j)/2 - D g.S, whatever the velocity along e."""
    x_i, x_j, e, n, S = axis_edge(2.0 ** -15, 0.0, 2e-5)
    V = (250.0 * e + 40.0 * n)[None, :]
    g = np.array([[1e18, -3e18]])
    u_i, u_j = np.array([2e16]), np.array([5e16])
    F = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, V, 0.1, g)
    Sv = S[0]
    expect = (V[0] @ Sv) * 0.5 * (u_i[0] + u_j[0]) - 0.1 * (g[0] @ Sv)
    assert abs(F[0] - expect) <= 1e-13 * abs(expect)


def test_limits_upwind_and_pure_diffusion():
    h = 2.0 ** -17
    x_i, x_j, e, n, S = axis_edge(h, 2e-5, 0.0)
    u_i, u_j = np.array([7e15]), np.array([2e15])
    for Vt in (300.0, -300.0):
        V = (Vt * e)[None, :]
        up = (u_i if Vt > 0 else u_j)[0]
        F0 = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, V, 0.0, np.zeros((1, 2)))
        assert F0[0] == pytest.approx(Vt * 2e-5 * up, rel=1e-15)
        # strong drift: a = h V / D = 3e5 -> the same upwind value
        Fs = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, V, 1e-8, np.zeros((1, 2)))
        assert Fs[0] == pytest.approx(Vt * 2e-5 * up, rel=1e-12)
    # no drift: the two-point diffusion flux -D (u_j - u_i)/h (S.e)
    Fd = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, np.zeros((1, 2)), 0.1, np.zeros((1, 2)))
    assert Fd[0] == pytest.approx(-0.1 * (u_j[0] - u_i[0]) / h * 2e-5, rel=1e-14)


def test_antisymmetric_under_edge_reversal():
    rng = np.random.Generator(np.random.PCG64(5))
    x_i = rng.normal(size=(50, 2)) * 1e-4
    x_j = x_i + rng.normal(size=(50, 2)) * 2e-5
    S = rng.normal(size=(50, 2)) * 1e-5
    V = rng.normal(size=(50, 2)) * 1e3
    g = rng.normal(size=(50, 2)) * 1e18
    u_i, u_j = rng.uniform(1e12, 1e18, 50), rng.uniform(1e12, 1e18, 50)
    F = O.sg_edge_flux(u_i, u_j, x_i, x_j, S, V, 0.1, g)
    Fr = O.sg_edge_flux(u_j, u_i, x_j, x_i, -S, V, 0.1, g)
    np.testing.assert_allclose(Fr, -F, rtol=1e-13, atol=1e-13 * np.abs(F).max())


def _sg(problem):
    problem.opts.scheme = W.FLUX_SG
    return problem


def test_sg_step_uniform_state_and_charge_ledger():
    """A uniform neutral state in the uniform field of the plates is preserved; with a
    Gaussian seed and Townsend ionisation the charge changes only by the boundary ledger."""
    q = _sg(W.plates_problem(13, 11, 1e-2, 0.8e-2, 5e3, seed=3, n_peak=0.0, n_back=1e12))
    oq = O.Oracle(q)
    m = oq.initial_state()
    for _ in range(3):
        m, _ = oq.step(m)
    for s in range(2):
        np.testing.assert_allclose(m[s], 1e12, rtol=1e-12)
    for axisym in (False, True):
        if axisym:
            p = _sg(W.axisym_problem(17, 13, 1e-2, 0.6e-2, 2e4, seed=4, source=W.SRC_TOWNSEND,
                                     field_dependent=True))
        else:
            p = _sg(W.plates_problem(17, 15, 1e-2, 1e-2, 2e4, seed=4, source=W.SRC_TOWNSEND,
                                     field_dependent=True))
        o = O.Oracle(p)
        n = o.initial_state()
        scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n)
        for _ in range(6):
            Q0 = o.charge(n)
            n, info = o.step(n)
            ledger = sum(-info["dt"] * O.E_CHARGE * sp_.charge * (info["outflow"][s] - info["source_total"][s])
                         for s, sp_ in enumerate(p.species))
            assert abs(o.charge(n) - Q0 - ledger) <= 1e-13 * scale


def test_sg_differs_from_llw_only_through_the_flux():
    """Same problem, same first Poisson solve and time step; the densities after one step
    differ (the schemes differ) but by less than the seed's own scale."""
    a = W.plates_problem(15, 15, 1e-2, 1e-2, 1e4, seed=8)
    b = _sg(W.plates_problem(15, 15, 1e-2, 1e-2, 1e4, seed=8))
    oa, ob = O.Oracle(a), O.Oracle(b)
    na, ia = oa.step(oa.initial_state())
    nb, ib = ob.step(ob.initial_state())
    assert ia["dt"] == ib["dt"]
    np.testing.assert_array_equal(ia["phi"], ib["phi"])
    d = np.abs(na[0] - nb[0]).max() / np.abs(na[0]).max()
    assert 0.0 < d < 0.1
