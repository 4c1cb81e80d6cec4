"""Pins of the oracle's photoionisation source (three-term Helmholtz fit of the streamer
benchmark's third case): each Helmholtz term against the closed-form solution of the
one-dimensional problem between two grounded plates (planar and axisymmetric), converging at
second order; linearity and the sum over terms; the step adds S_ph to electrons and positive
ions only; the charge ledger closes.  CPU only."""
import numpy as np
import pytest

import avip_oracle as O
from paper_2201_01291_gb300 import workloads as W


def closed_form(y, L, a, kap, I):
    """-S'' + kap^2 S = a I on (0, L), S(0) = S(L) = 0."""
    return a * I / kap ** 2 * (1.0 - np.cosh(kap * (y - 0.5 * L)) / np.cosh(0.5 * kap * L))


@pytest.mark.parametrize("axisym", [False, True])
def test_helmholtz_terms_against_1d_closed_form(axisym):
    """Uniform photon production between two grounded electrodes, zero normal derivative on
    the other sides: every term is the 1D closed form in the inter-electrode coordinate."""
    ph = W.Photo([3.0e4, 2.0e5, 1.5e6], [400.0, 1500.0, 6000.0], 1.0)
    L = 2e-3
    I = 1e25
    errs = []
    for n in (11, 21, 41, 81):
        if axisym:
            p = W.axisym_problem(n, n // 2 + 1, L, 1e-3, 0.0, seed=4, n_peak=0.0, n_back=0.0)
            coord = p.xy[:, 0]
        else:
            p = W.plates_problem(n // 2 + 1, n, 1e-3, L, 0.0, seed=4, n_peak=0.0, n_back=0.0)
            coord = p.xy[:, 1]
        p = W.dataclasses.replace(p, photo=ph)
        o = O.Oracle(p)
        S, terms = o.photo_source(np.full(p.n_nodes, I))
        e = 0.0
        for j in range(3):
            ref = closed_form(coord, L, ph.a[j], ph.kappa[j], I)
            e = max(e, np.abs(terms[j] - ref).max() / np.abs(ref).max())
        errs.append(e)
        np.testing.assert_allclose(S, terms[0] + terms[1] + terms[2], rtol=1e-15)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3 and rates[-2:].mean() > 1.7, (errs, rates)


def test_linearity_and_positivity():
    p = W.plates_problem(21, 19, 1e-2, 1e-2, 2e4, seed=3, field_dependent=True, source=W.SRC_TOWNSEND)
    p = W.dataclasses.replace(p, photo=W.photo_air())
    o = O.Oracle(p)
    I = W.gaussian(p.xy, 5e-3, 5e-3, 1e-3, 1e26, 0.0)
    S1, t1 = o.photo_source(I)
    S2, _ = o.photo_source(2.5 * I)
    np.testing.assert_allclose(S2, 2.5 * S1, rtol=1e-12, atol=1e-12 * np.abs(S2).max())
    assert S1.max() > 0 and S1[p.node_bc == 1].max() == 0.0
    # the long-range term spreads further than the short-range one
    far = np.hypot(p.xy[:, 0] - 5e-3, p.xy[:, 1] - 5e-3) > 3e-3
    assert (t1[0][far].sum() / t1[0].sum()) > (t1[2][far].sum() / t1[2].sum())


def test_step_adds_photo_to_electrons_and_positive_ions_only():
    """Same state and fixed dt with and without photoionisation: the difference of the
    updated densities is dt S_ph for electrons and positive ions, zero for negative ions."""
    base = W.plates_problem(25, 23, 1e-2, 1e-2, 2.5e4, seed=5, field_dependent=True,
                            source=W.SRC_TOWNSEND_ATTACH, n_species=3)
    with_ph = W.dataclasses.replace(base, photo=W.photo_air())
    o0, o1 = O.Oracle(base), O.Oracle(with_ph)
    n = o0.initial_state()
    dt = 1e-12
    a, _ = o0.step(n, dt_fixed=dt)
    b, info = o1.step(n, dt_fixed=dt)
    S = o1.last_photo
    assert S.max() > 0
    for s in (0, 1):
        np.testing.assert_allclose(b[s] - a[s], dt * S, rtol=1e-6, atol=1e-9 * np.abs(a[s]).max())
    np.testing.assert_array_equal(b[2], a[2])


def test_photo_charge_ledger():
    p = W.plates_problem(21, 19, 1e-2, 1e-2, 2.5e4, seed=2, field_dependent=True, source=W.SRC_TOWNSEND)
    p = W.dataclasses.replace(p, photo=W.photo_air())
    o = O.Oracle(p)
    n = o.initial_state()
    scale = sum(O.E_CHARGE * np.sum(o.V_node * x) for x in n)
    for _ in range(5):
        Q0 = o.charge(n)
        n, info = o.step(n)
        ledger = sum(-info["dt"] * O.E_CHARGE * sp_.charge * (info["outflow"][s] - info["source_total"][s])
                     for s, sp_ in enumerate(p.species))
        assert abs(o.charge(n) - Q0 - ledger) <= 1e-13 * scale
