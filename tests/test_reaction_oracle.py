"""Pins of the reaction oracle (oracle/reaction.py): closed-form solutions of the linear
reaction, second-order convergence of the reaction-by-reaction splitting against a
high-accuracy solution of the ODE system (Eq. ode-system with Eq. fhn / Eq. a-p), fixed
points and the p = 0 limit of the QSS update."""
import math

import numpy as np
import pytest

from oracle import reaction as rx

scipy_integrate = pytest.importorskip("scipy.integrate")

FN_PARAMS = rx.Reaction(model=rx.FN, a=0.1, eps0=0.08, beta=1.0, gamma=1.0, sigma=0.0)
AP_PARAMS = rx.Reaction(model=rx.AP, a=0.15, b=0.15, k=8.0, eps0=0.002, mu1=0.2, mu2=0.3)


def test_fn_gate_reaction_is_the_exact_exponential():
    # with V frozen, dw/dt = eps0 (beta V - gamma w - sigma) relaxes exponentially to
    # (beta V - sigma)/gamma with rate eps0 gamma
    r = rx.Reaction(model=rx.FN, a=0.1, eps0=0.3, beta=0.7, gamma=1.3, sigma=0.05)
    V = np.array([0.0, 0.4, 1.0]); w = np.array([0.2, -0.1, 0.5]); t = 0.9
    winf = (r.beta * V - r.sigma) / r.gamma
    exact = winf + (w - winf) * math.exp(-r.eps0 * r.gamma * t)
    np.testing.assert_allclose(rx.reaction_w(V, w, r, t), exact, rtol=1e-14, atol=1e-15)


def test_qss_limit_at_zero_loss_rate():
    # FN at V = a has p = 0: the update is the explicit step V + dt q
    r = FN_PARAMS
    V = np.array([r.a]); w = np.array([0.3])
    np.testing.assert_allclose(rx.reaction_V(V, w, r, 0.2), r.a - 0.2 * 0.3, rtol=1e-15)
    # and it is continuous through p = 0
    near = rx.qss(1.0, 0.5, 1e-9, 0.2)
    assert abs(near - rx.qss(1.0, 0.5, 0.0, 0.2)) < 1e-9


@pytest.mark.parametrize("r", [FN_PARAMS, AP_PARAMS])
def test_rest_state_is_a_fixed_point(r):
    V, w = np.zeros(3), np.zeros(3)
    for _ in range(10):
        V, w = rx.reaction_step(V, w, r, 0.1)
    assert np.all(V == 0.0) and np.all(w == 0.0)


def _reference(r, V0, w0, T):
    sol = scipy_integrate.solve_ivp(lambda t, y: rx.rhs(y[0], y[1], r), (0.0, T), [V0, w0],
                                    method="DOP853", rtol=1e-12, atol=1e-14)
    return sol.y[0, -1], sol.y[1, -1]


def _run(step, r, V0, w0, T, dt):
    V, w = np.array([V0]), np.array([w0])
    for _ in range(int(round(T / dt))):
        V, w = step(V, w, r, dt)
    return V[0], w[0]


def _lie(V, w, r, dt, flow_V, flow_w):
    # a planted first-order composition: R_V(dt) then R_w(dt)
    V = flow_V(V, w, r, dt)
    return V, flow_w(V, w, r, dt)


def _exact_V(V, w, r, t):
    # the V reaction with w frozen, solved to 1e-13
    f = lambda s, y: [rx.rhs(y[0], w[0], r)[0]]
    return np.array([scipy_integrate.solve_ivp(f, (0.0, t), [V[0]], method="DOP853",
                                               rtol=1e-13, atol=1e-15).y[0, -1]])


def _exact_w(V, w, r, t):
    f = lambda s, y: [rx.rhs(V[0], y[0], r)[1]]
    return np.array([scipy_integrate.solve_ivp(f, (0.0, t), [w[0]], method="DOP853",
                                               rtol=1e-13, atol=1e-15).y[0, -1]])


CASES = [(FN_PARAMS, 0.3, 0.0, 5.0), (AP_PARAMS, 0.5, 0.1, 2.0)]


@pytest.mark.parametrize("r,V0,w0,T", CASES)
def test_composition_is_second_order_with_exact_subflows(r, V0, w0, T):
    ref = np.array(_reference(r, V0, w0, T))
    strang = lambda V, w, r, dt: rx.reaction_step(V, w, r, dt, _exact_V, _exact_w)
    lie = lambda V, w, r, dt: _lie(V, w, r, dt, _exact_V, _exact_w)
    e = [np.max(np.abs(np.array(_run(strang, r, V0, w0, T, dt)) - ref)) for dt in (0.1, 0.05)]
    assert 3.5 < e[0] / e[1] < 4.5
    # the planted first-order composition converges at first order only
    el = [np.max(np.abs(np.array(_run(lie, r, V0, w0, T, dt)) - ref)) for dt in (0.1, 0.05)]
    assert 1.7 < el[0] / el[1] < 2.3


@pytest.mark.parametrize("r,V0,w0,T", CASES)
def test_qss_scheme_converges_at_first_order(r, V0, w0, T):
    # the QSS update freezes p and q at the start of each reaction: first order overall
    ref = np.array(_reference(r, V0, w0, T))
    e = [np.max(np.abs(np.array(_run(rx.reaction_step, r, V0, w0, T, dt)) - ref))
         for dt in (0.02, 0.01, 0.005)]
    assert e[0] < 5e-3
    assert 1.8 < e[0] / e[1] < 2.2 and 1.8 < e[1] / e[2] < 2.2
