"""Pins of the frozen-geometry reading (R11) in the oracle: pair vectors kept from the
configuration update instead of recomputed at every half step.

Where positions do not move relative to one another over a half step, both readings must
give the same result; over a whole step the frozen pair terms stay antisymmetric, so
momentum is conserved; and the difference between the readings shrinks with the step."""
import numpy as np
import pytest

from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import perturbed_state


def _state(prob, x, v, rho, drho):
    st, w = o.state_from_problem(prob)
    st.x, st.v, st.rho, st.drho = x.copy(), v.copy(), rho.copy(), drho.copy()
    return st, w


def _jittered_tank():
    prob = wk.dam_break(dim=2, H=0.3, L=0.4, dp=0.02, tank=1.0)
    x, _, rho, drho = perturbed_state(prob, 3, 0.0, 0.01)
    x = x + np.random.default_rng(4).uniform(-0.1, 0.1, x.shape) * prob.dp
    return prob, x, rho, drho


def test_at_rest_the_first_half_step_is_the_same_in_both_readings():
    # v = 0: the mid-point positions are the configuration's, fluid and wall pairs alike
    prob, x, rho, drho = _jittered_tank()
    prm = o.Params.from_problem(prob)
    st, w = _state(prob, x, np.zeros_like(x), rho, drho)
    nb = o.neighbour_sets(st.x, w.x, prm)
    geo = o.frozen_geometry(st, w, nb, prm)
    dt = 0.2 * o.dt_acoustic(st.v, prm)
    acc0 = np.zeros_like(x)
    _, a_rec = o.pressure_relaxation(st, w, nb, acc0, dt, prm)
    _, a_frz = o.pressure_relaxation(st, w, nb, acc0, dt, prm, geo)
    assert np.abs(a_rec - prm.gravity).max() > 1.0          # the pair forces are not trivial
    np.testing.assert_allclose(a_frz, a_rec, rtol=0, atol=1e-12 * np.abs(a_rec).max())


def test_uniform_translation_keeps_pair_vectors_in_the_density_relaxation():
    # one velocity for every particle in a periodic box: r_i - r_j never changes
    prob = wk.periodic_box(dim=2, n=20, seed=5, vel_amp=0.0, rho_amp=0.02)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    st.v[:] = np.array([0.7, -0.4])
    st.drho = np.random.default_rng(6).uniform(-0.1, 0.1, st.rho.shape)
    nb = o.neighbour_sets(st.x, w.x, prm)
    geo = o.frozen_geometry(st, w, nb, prm)
    dt = o.dt_acoustic(st.v, prm)
    rec = o.density_relaxation(st, w, nb, dt, prm)
    frz = o.density_relaxation(st, w, nb, dt, prm, geo)
    assert np.abs(rec.drho).max() > 1e-3
    np.testing.assert_allclose(frz.drho, rec.drho, rtol=0, atol=1e-10 * np.abs(rec.drho).max())
    np.testing.assert_array_equal(frz.x, rec.x)


def test_frozen_geometry_is_antisymmetric_and_conserves_momentum():
    prob = wk.periodic_box(dim=2, n=24, seed=7, vel_amp=0.3, rho_amp=0.02)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    nb = o.neighbour_sets(st.x, w.x, prm)
    I, J = nb[0], nb[1]
    rij = o.frozen_geometry(st, w, nb, prm)[0]
    # (i, j) and (j, i) carry opposite vectors
    pos = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(I, J))}
    back = np.array([pos[(int(b), int(a))] for a, b in zip(I, J)])
    np.testing.assert_array_equal(rij[back], -rij)
    p0 = o.diagnostics(st, prm)["momentum"]
    out, info = o.advection_step(st, w, prm, frozen=True)
    p1 = o.diagnostics(out, prm)["momentum"]
    scale = np.sum(st.m * np.linalg.norm(st.v, axis=1))
    assert info.substeps >= 3
    assert np.abs(p1 - p0).max() <= 1e-13 * scale


def test_readings_differ_by_a_first_order_term_in_the_step():
    # the frozen and recomputed readings part at O(dt): halving dt about halves the gap
    prob, x, rho, drho = _jittered_tank()
    prm = o.Params.from_problem(prob)
    rng = np.random.default_rng(8)
    v = rng.uniform(-0.3, 0.3, x.shape)
    st, w = _state(prob, x, v, rho, drho)
    nb = o.neighbour_sets(st.x, w.x, prm)
    geo = o.frozen_geometry(st, w, nb, prm)
    acc0 = np.zeros_like(x)
    gaps = []
    for dt in (2e-4, 1e-4, 5e-5):
        _, a_rec = o.pressure_relaxation(st, w, nb, acc0, dt, prm)
        _, a_frz = o.pressure_relaxation(st, w, nb, acc0, dt, prm, geo)
        gaps.append(np.abs(a_frz - a_rec).max())
    assert gaps[0] > 0
    assert 1.8 < gaps[0] / gaps[1] < 2.2 and 1.8 < gaps[1] / gaps[2] < 2.2


def test_planted_sign_flip_of_the_frozen_vectors_is_caught(monkeypatch):
    orig = o.frozen_geometry
    monkeypatch.setattr(o, "frozen_geometry", lambda st, w, nb, prm: tuple(-g for g in orig(st, w, nb, prm)))
    with pytest.raises(AssertionError):
        test_at_rest_the_first_half_step_is_the_same_in_both_readings()
