"""Plain FP64 CPU oracle of the reaction step of reaction-diffusion (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use this
module. It shares no code with the CUDA library.

The method (paper Sec. "SPH method for reaction-diffusion" and "Reaction-by-reaction
splitting"), per particle, in the paper's order:

  * Operator splitting separates the diffusion of V (Eq. diffusion, oracle/diffusion.py)
    from the ODE system dV/dt = I(V, w), dw/dt = g(V, w) (Eq. ode-system).
  * I and g: the FitzHugh-Nagumo model (Eq. fhn) or the Aliev-Panfilov model (Eq. a-p).
  * Second-order reaction-by-reaction splitting (Eq. ode-spliting-2rd): a step of length dt
    applies R_V(dt/2), then R_w(dt/2), then R_w(dt/2), then R_V(dt/2), each reaction
    advancing one variable with the other held fixed.
  * Each reaction is written dy/dt = q(y) - p(y) y (Eq. ode-new-form) and advanced by the
    quasi-steady-state update y' = y e^(-p dt) + (q/p)(1 - e^(-p dt)) with p and q taken at
    the reaction's starting value (Eq. ode-qss).

Readings where the paper is silent:
  R16 The production/loss split of each right-hand side, chosen so that q does not depend
      on the reacting variable where the model allows:
        FN  R_V: q = -w,                    p = (V - a)(V - 1)
            R_w: q = eps0 (beta V - sigma), p = eps0 gamma
        AP  R_V: q = 0,                     p = k (V - a)(V - 1) + w
            R_w: q = -eps k V (V - b - 1),  p = eps,  eps = eps0 + mu1 w / (mu2 + V)
      (for FN's R_w, p and q do not depend on w, so the update is exact for the frozen V).
      p may be zero or negative; (1 - e^(-p dt))/p is evaluated as
      -expm1(-p dt)/p and taken as dt when |p dt| < 1e-12. The model parameters are the
      caller's (the paper gives none).

Order: the composition is second order with exact sub-flows, but the QSS update freezes
p and q at the start of each reaction, so where p depends on the reacting variable (FN's and
AP's R_V, AP's R_w) it is first-order accurate, and so is the whole step.

Parity pins: tests/test_reaction_oracle.py (the closed-form exponential solution of the
linear reaction, second-order convergence of the composition with exact sub-flows and
first-order convergence of the QSS scheme against a high-accuracy ODE solution, a planted
first-order composition, fixed points, the p = 0 limit). None is unpinned.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FN, AP = 1, 2


@dataclass
class Reaction:
    model: int            # FN or AP
    a: float = 0.0
    b: float = 0.0        # AP
    k: float = 0.0        # AP
    eps0: float = 0.0
    mu1: float = 0.0      # AP
    mu2: float = 0.0      # AP
    beta: float = 0.0     # FN
    gamma: float = 0.0    # FN
    sigma: float = 0.0    # FN


def qss(y, q, p, dt):
    """Eq. ode-qss: y e^(-p dt) + q (1 - e^(-p dt))/p, with the p -> 0 limit (R16)."""
    y, q, p = np.asarray(y, float), np.asarray(q, float), np.asarray(p, float)
    x = -p * dt
    small = np.abs(x) < 1e-12
    frac = np.where(small, dt, -np.expm1(x) / np.where(small, 1.0, p))
    return y * np.exp(x) + q * frac


def reaction_V(V, w, r: Reaction, dt):
    """R_V(dt): V advanced with w held fixed (R16)."""
    if r.model == FN:
        return qss(V, -w, (V - r.a) * (V - 1.0), dt)
    return qss(V, np.zeros_like(V), r.k * (V - r.a) * (V - 1.0) + w, dt)


def reaction_w(V, w, r: Reaction, dt):
    """R_w(dt): w advanced with V held fixed (R16)."""
    if r.model == FN:
        return qss(w, r.eps0 * (r.beta * V - r.sigma), np.full_like(w, r.eps0 * r.gamma), dt)
    eps = r.eps0 + r.mu1 * w / (r.mu2 + V)
    return qss(w, -eps * r.k * V * (V - r.b - 1.0), eps, dt)


def reaction_step(V, w, r: Reaction, dt, flow_V=None, flow_w=None):
    """Eq. ode-spliting-2rd: R_V(dt/2), R_w(dt/2), R_w(dt/2), R_V(dt/2), in that order.
    flow_V / flow_w replace the QSS reactions (the pins pass exact sub-flows to check the
    composition on its own)."""
    fV = flow_V or reaction_V
    fw = flow_w or reaction_w
    h = 0.5 * dt
    V = fV(V, w, r, h)
    w = fw(V, w, r, h)
    w = fw(V, w, r, h)
    V = fV(V, w, r, h)
    return V, w


def rhs(V, w, r: Reaction):
    """I(V, w) and g(V, w) of Eq. fhn / Eq. a-p (for the pins' reference solutions)."""
    if r.model == FN:
        return -V * (V - r.a) * (V - 1.0) - w, r.eps0 * (r.beta * V - r.gamma * w - r.sigma)
    eps = r.eps0 + r.mu1 * w / (r.mu2 + V)
    return -r.k * V * (V - r.a) * (V - 1.0) - w * V, eps * (-r.k * V * (V - r.b - 1.0) - w)
