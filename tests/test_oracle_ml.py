"""Pins of the oracle's three-species air chemistry (section "Hyperbole electrodes": ionisation,
field-dependent attachment, electron-ion and ion-ion recombination, immobile ions) and of the
linear electrode-voltage ramp (Fig. pin-pin_anode_time).  Closed forms written from the
governing equations, not from the oracle: the sources conserve charge pointwise; a uniform
neutral state without field evolves by the forward-Euler recombination ODE; interior nodes
of a uniform state in a uniform field evolve by the local ionisation/attachment/recombination
ODE; the potential of a charge-free gap follows the ramp exactly.  CPU only."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


def ml(nx=15, ny=13, Lx=5e-3, Ly=5e-3, v_max=5e3, **kw):
    return W.morrow_lowke_problem(nx, ny, Lx, Ly, v_max, seed=3, **kw)


def test_sources_conserve_charge_pointwise():
    p = ml()
    rng = np.random.default_rng(0)
    o = O.Oracle(p)
    n = [rng.uniform(1e14, 1e18, p.n_nodes) for _ in range(3)]
    Emag = rng.uniform(0.0, 3e7, p.n_nodes)
    mu = [O.mobility(sp_, Emag) for sp_ in p.species]
    S = o.sources(n, Emag, mu)
    q = [sp_.charge for sp_ in p.species]
    net = sum(q[s] * S[s] for s in range(3))
    scale = sum(np.abs(S[s]) for s in range(3))
    assert np.all(np.abs(net) <= 1e-14 * scale)


def test_source_closed_form_at_one_point():
    """S_e = (alpha - eta) mu_e E n_e - beta n_e n_p, S_p = alpha mu_e E n_e - beta n_e n_p
    - beta n_n n_p, S_n = eta mu_e E n_e - beta n_n n_p, with alpha and eta from their fits."""
    p = ml()
    A, B, A_eta, B_eta, beta_r = p.source.params
    o = O.Oracle(p)
    E = 1.2e7
    ne, npos, nneg = 3e17, 5e17, 2e17
    n = [np.full(p.n_nodes, v) for v in (ne, npos, nneg)]
    Emag = np.full(p.n_nodes, E)
    mu = [O.mobility(sp_, Emag) for sp_ in p.species]
    mu_e = p.species[0].mob_params[0] * (E / p.species[0].mob_params[1]) ** p.species[0].mob_params[2]
    alpha = A * np.exp(-B / E)
    eta = A_eta * np.exp(-B_eta / E)
    w = mu_e * E
    S = o.sources(n, Emag, mu)
    np.testing.assert_allclose(S[0][0], (alpha - eta) * w * ne - beta_r * ne * npos, rtol=1e-13)
    np.testing.assert_allclose(S[1][0], alpha * w * ne - beta_r * ne * npos - beta_r * nneg * npos, rtol=1e-13)
    np.testing.assert_allclose(S[2][0], eta * w * ne - beta_r * nneg * npos, rtol=1e-13)


def test_recombination_ode_without_field():
    """v_max = 0 and a uniform neutral state (n_p = n_e + n_n): no field, no transport, so
    every node follows forward Euler of dn_e/dt = -beta n_e n_p, dn_p/dt = -beta (n_e + n_n) n_p,
    dn_n/dt = -beta n_n n_p, with the time step of the dielectric / chemical / Fourier limits."""
    p = ml(v_max=0.0, n_back=4e17)
    ne0, nn0 = 4e17, 1e17
    p.species[0].n0[:] = ne0
    p.species[2].n0[:] = nn0
    p.species[1].n0[:] = ne0 + nn0
    beta_r = p.source.params[4]
    o = O.Oracle(p)
    n = o.initial_state()
    t = 0.0
    for _ in range(4):
        e, pos, neg = n[0][0], n[1][0], n[2][0]
        new, info = o.step(n, t=t)
        dt = info["dt"]
        # the time-step candidates, written out: dielectric (only electrons move), chemical,
        # Fourier on the shortest side of the mesh
        mu_e = p.species[0].mob_params[0] * (p.species[0].mob_params[3] / p.species[0].mob_params[1]) ** \
            p.species[0].mob_params[2]
        dt_diel = p.opts.a_diel * O.EPS0 / (O.E_CHARGE * e * mu_e)
        dt_chem = p.opts.a_chem * e / (beta_r * e * pos)
        dx = min(o.dx_tau)
        dt_four = p.opts.fourier * dx ** 2 / p.species[0].D
        np.testing.assert_allclose(dt, min(dt_diel, dt_chem, dt_four), rtol=1e-12)
        for s, S in enumerate((-beta_r * e * pos, -beta_r * pos * (e + neg), -beta_r * neg * pos)):
            np.testing.assert_allclose(new[s], n[s][0] + dt * S, rtol=1e-13, atol=0.0)
        n = new
        t += dt


def test_uniform_field_interior_ode():
    """Plates at 30 kV over 5 mm (6 MV/m), uniform densities: at interior nodes the edge fluxes
    cancel (uniform u and V), so one step is forward Euler of the local chemistry with
    |E| = V/L, the power-law mobility and the two Arrhenius-form fits."""
    p = ml(v_max=3e4, v_rise=0.0, n_back=1e16, jitter=0.2)
    p.species[2].n0[:] = 2e15
    p.species[1].n0[:] = 1.2e16
    o = O.Oracle(p)
    n = o.initial_state()
    new, info = o.step(n)
    E = 3e4 / 5e-3
    A, B, A_eta, B_eta, beta_r = p.source.params
    m = p.species[0].mob_params
    w = m[0] * (E / m[1]) ** m[2] * E
    alpha, eta = A * np.exp(-B / E), A_eta * np.exp(-B_eta / E)
    ne, npos, nneg = 1e16, 1.2e16, 2e15
    S = ((alpha - eta) * w * ne - beta_r * ne * npos, alpha * w * ne - beta_r * (ne + nneg) * npos,
         eta * w * ne - beta_r * nneg * npos)
    interior = ~o.is_bnd
    for s in range(3):
        np.testing.assert_allclose(new[s][interior], n[s][interior] + info["dt"] * S[s], rtol=1e-9)


@pytest.mark.parametrize("frac", [0.25, 0.5, 1.0, 1.5])
def test_voltage_ramp_linear_potential(frac):
    """A charge-free gap: phi(t) = min(t / v_rise, 1) V y / L exactly."""
    p = ml(v_max=5e3, v_rise=2e-9, n_back=0.0)
    o = O.Oracle(p)
    n = [np.zeros(p.n_nodes) for _ in range(3)]
    t = frac * 2e-9
    phi = o.poisson(n, t)
    np.testing.assert_allclose(phi, min(frac, 1.0) * 5e3 * p.xy[:, 1] / 5e-3, rtol=1e-12, atol=1e-9)


def test_run_follows_the_ramp_and_ledger_closes():
    """run() evaluates step k's potential at t_k = sum of the earlier steps (the linear
    potential scaled by the ramp when the gap is charge free); the charge ledger closes with
    the chemistry on."""
    p = ml(v_max=5e3, v_rise=2e-9, n_back=0.0)
    o = O.Oracle(p)
    n = [np.zeros(p.n_nodes) for _ in range(3)]
    t = 0.0
    for k in range(3):
        n, info = o.step(n, dt_fixed=3e-10, t=t)
        np.testing.assert_allclose(info["phi"], min(t / 2e-9, 1.0) * 5e3 * p.xy[:, 1] / 5e-3, atol=1e-9)
        t += info["dt"]
    q = ml(nx=21, ny=19, v_max=2e4, v_rise=1e-10, n_back=1e16)
    q.species[0].n0[:] = W.gaussian(q.xy, 2.5e-3, 2.5e-3, 5e-4, 1e19, 1e16)
    q.species[1].n0[:] = q.species[0].n0
    oq = O.Oracle(q)
    m = oq.initial_state()
    scale = sum(O.E_CHARGE * np.sum(oq.V_node * x) for x in m)
    t = 0.0
    for _ in range(5):
        Q0 = oq.charge(m)
        m, info = oq.step(m, t=t)
        t += info["dt"]
        ledger = sum(-info["dt"] * O.E_CHARGE * sp_.charge * (info["outflow"][s] - info["source_total"][s])
                     for s, sp_ in enumerate(q.species))
        assert abs(oq.charge(m) - Q0 - ledger) <= 1e-13 * scale
