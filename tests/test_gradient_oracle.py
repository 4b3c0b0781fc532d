"""Pins of the oracle's particle gradients (Eqs. gradsph-strong, gradsph-weak; reading R18).

What fixes them independently of the code:
  * the continuum identity int (-dW/dr / r) x_a x_b dV = delta_ab (quadrature), so on a
    lattice both forms reproduce the gradient of a linear field in the interior, with an
    error that falls to zero as h/dp grows;
  * the strong form of a constant field is exactly zero, everywhere (zero-order
    consistency); the weak form is zero only where the support is full;
  * the weak form is antisymmetric per pair: sum_i V_i grad f_i = 0 in a periodic box;
  * a still tank with the hydrostatic pressure p = rho0 g (H - y): the wall problem's
    extrapolated values (R4) carry the strong-form gradient rho0 g up to the wall;
  * a double loop over every pair of a tiny set, written out.
Planted mistakes (a flipped kernel derivative, the sum in place of the difference, m_j in
place of V_j, the wall extrapolation with the wrong sign) each fail one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk

RHO0 = 1000.0          # far from 1, so that m_j and V_j = m_j / rho_j differ


class _Block:
    """A lattice block of n^d particles in the unit cube, no walls (its faces are free
    surfaces), h = hdp dp."""

    def __init__(self, d, n, hdp):
        self.dim, self.dp = d, 1.0 / n
        self.h = hdp * self.dp
        self.rho0, self.c0, self.cfl_ad, self.cfl_ac, self.u_ref, self.nu = RHO0, 10.0, 0.25, 0.6, 1.0, 0.0
        self.gravity = np.zeros(3)
        self.lo, self.hi = np.full(3, -0.5), np.full(3, 1.5)
        self.periodic = np.zeros(3, dtype=int)
        self.free_surface = 1
        ax = (np.arange(n) + 0.5) * self.dp
        g = np.meshgrid(*([ax] * d), indexing="ij")
        self.x = np.stack([gg.ravel() for gg in g], axis=1)


def _state(blk, rho):
    x = blk.x
    return o.State(x, np.zeros_like(x), rho, np.zeros(len(x)), rho * blk.dp ** blk.dim)


def _no_walls(d):
    return o.Walls(np.zeros((0, d)), np.zeros((0, d)), np.zeros(0))


def _linear_errors(d, n, hdp):
    blk = _Block(d, n, hdp)
    prm = o.Params.from_problem(blk)
    a = np.array([0.3, -0.7, 0.2])[:d]
    rho = RHO0 * (1.0 + 1e-3 * (blk.x @ a))            # V_j = dp^d exactly
    st = _state(blk, rho)
    w = _no_walls(d)
    gr = o.gradients(st, w, o.neighbour_sets(st.x, w.x, prm), prm)
    inner = np.all((blk.x > 2.05 * prm.h) & (blk.x < 1.0 - 2.05 * prm.h), axis=1)
    assert inner.sum() > 50
    exact = RHO0 * 1e-3 * a
    err = lambda g: np.max(np.abs(g[inner] - exact)) / np.linalg.norm(exact)
    # pressure: p = c0^2 (rho - rho0), so grad p = c0^2 grad rho in the interior
    errp = np.max(np.abs(gr["p_strong"][inner] - prm.c0 ** 2 * exact)) / (prm.c0 ** 2 * np.linalg.norm(exact))
    return err(gr["rho_strong"]), err(gr["rho_weak"]), errp


def test_continuum_moment_identity():
    for d in (2, 3):
        shell = (lambda r: 2 * math.pi * r) if d == 2 else (lambda r: 4 * math.pi * r * r)
        val = integrate.quad(lambda r: -o.kernel_dW(r, 1.0, d) / r * r * r / d * shell(r), 0.0, 2.0)[0]
        assert abs(val - 1.0) < 1e-12


def test_linear_field_gradient_converges_to_the_exact_one():
    e2 = [_linear_errors(2, 40, hdp) for hdp in (1.3, 2.0, 4.0)]
    e3 = [_linear_errors(3, 16, hdp) for hdp in (1.3, 2.0)]
    for es in (e2, e3):
        for k in range(3):
            seq = [e[k] for e in es]
            assert all(b < a for a, b in zip(seq, seq[1:])), seq
    assert max(e2[0]) < 0.03 and max(e3[0]) < 0.03       # h = 1.3 dp: a few percent
    assert max(e2[2]) < 1e-5                               # h = 4 dp, 2D
    assert max(e3[1]) < 1e-3                               # h = 2 dp, 3D


def test_constant_field():
    blk = _Block(2, 24, 1.3)
    prm = o.Params.from_problem(blk)
    st = _state(blk, np.full(len(blk.x), RHO0 * 1.01))
    w = _no_walls(2)
    gr = o.gradients(st, w, o.neighbour_sets(st.x, w.x, prm), prm)
    scale = RHO0 / prm.h
    assert np.max(np.abs(gr["rho_strong"])) < 1e-12 * scale     # everywhere, surface included
    assert np.max(np.abs(gr["p_strong"])) < 1e-12 * scale * prm.c0 ** 2
    inner = np.all((blk.x > 2.05 * prm.h) & (blk.x < 1.0 - 2.05 * prm.h), axis=1)
    assert np.max(np.abs(gr["rho_weak"][inner])) < 1e-10 * scale
    assert np.max(np.abs(gr["rho_weak"][~inner])) > 0.1 * scale   # truncated support


def test_weak_form_is_antisymmetric_per_pair():
    prob = wk.periodic_box(dim=2, n=24, seed=4, vel_amp=0.0, rho_amp=0.05)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    st.rho = prm.rho0 * (1.0 + np.random.default_rng(8).uniform(-0.05, 0.05, st.x.shape[0]))
    gr = o.gradients(st, w, o.neighbour_sets(st.x, w.x, prm), prm)
    V = st.m / st.rho
    for k in ("rho_weak", "p_weak"):
        tot = np.sum(V[:, None] * gr[k], axis=0)
        assert np.all(np.abs(tot) < 1e-12 * np.sum(np.abs(V[:, None] * gr[k]), axis=0)), k


def _hydrostatic_errors():
    prob = wk.still_tank(dim=2, H=0.5, dp=0.0125)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    H = prob.meta["H"]
    g = -prm.gravity[1]
    p = prm.rho0 * g * (H - st.x[:, 1])
    st.rho = prm.rho0 + p / prm.c0 ** 2
    gr = o.gradients(st, w, o.neighbour_sets(st.x, w.x, prm), prm)
    below = st.x[:, 1] < H - 2.05 * prm.h                 # full support apart from the walls
    near_wall = below & ((st.x[:, 1] < 2.05 * prm.h) | (st.x[:, 0] < st.x[:, 0].min() + 2.05 * prm.h))
    assert near_wall.sum() > 20
    exact = np.array([0.0, -prm.rho0 * g])
    errs = {}
    for k in ("p_strong", "p_weak"):
        e = np.linalg.norm(gr[k][below] - exact, axis=1) / (prm.rho0 * g)
        errs[k] = (float(e.max()), float(e[near_wall[below]].max()))
    return errs


def test_hydrostatic_pressure_gradient_reaches_the_walls():
    # the strong form only: the weak form adds 2 p_i sum_j V_j grad_i W_ij, which is zero
    # only for uniform volumes, and here the fluid's V = m/rho (rho = rho0 + p/c0^2, 1 %
    # above rho0 at the floor) meets the walls' V_w = dp^d, an error that p_i amplifies by
    # (H - y)/h (about 30 % at the floor): the weak form serves conservation, not accuracy
    errs = _hydrostatic_errors()
    assert errs["p_strong"][0] < 0.05, errs
    assert errs["p_weak"][0] > 0.1, errs


def test_double_loop_on_a_tiny_set():
    prob = wk.dam_break(dim=2, H=0.2, L=0.2, dp=0.025)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    rng = np.random.default_rng(3)
    st.x = st.x + rng.uniform(-0.2, 0.2, st.x.shape) * prob.dp
    st.rho = prm.rho0 * (1.0 + rng.uniform(-0.02, 0.02, st.x.shape[0]))
    gr = o.gradients(st, w, o.neighbour_sets(st.x, w.x, prm), prm)
    N, d = st.x.shape
    c2 = prm.c0 ** 2
    p = c2 * (st.rho - prm.rho0)
    for i in range(N):
        acc = {k: np.zeros(d) for k in gr}
        for j in range(N):
            r = st.x[i] - st.x[j]
            dist = math.sqrt(r @ r)
            if j == i or dist >= 2 * prm.h:
                continue
            gW = o.kernel_dW(dist, prm.h, d) * r / dist
            Vj = st.m[j] / st.rho[j]
            acc["rho_strong"] += Vj * (st.rho[j] - st.rho[i]) * gW
            acc["rho_weak"] += Vj * (st.rho[i] + st.rho[j]) * gW
            acc["p_strong"] += Vj * (p[j] - p[i]) * gW
            acc["p_weak"] += Vj * (p[i] + p[j]) * gW
        for k in range(w.x.shape[0]):
            r = st.x[i] - w.x[k]
            dist = math.sqrt(r @ r)
            if dist >= 2 * prm.h:
                continue
            gW = o.kernel_dW(dist, prm.h, d) * r / dist
            pw = p[i] + st.rho[i] * ((w.x[k] - st.x[i]) @ prm.gravity)
            rw = prm.rho0 + pw / c2
            acc["rho_strong"] += w.V[k] * (rw - st.rho[i]) * gW
            acc["rho_weak"] += w.V[k] * (st.rho[i] + rw) * gW
            acc["p_strong"] += w.V[k] * (pw - p[i]) * gW
            acc["p_weak"] += w.V[k] * (p[i] + pw) * gW
        for key in gr:
            assert np.allclose(gr[key][i], acc[key], rtol=1e-10, atol=1e-9 * np.abs(acc[key]).max()), (i, key)


def test_planted_mistakes_are_caught(monkeypatch):
    orig = o.gradients
    # 1. flipped kernel derivative
    orig_dw = o.kernel_dW
    monkeypatch.setattr(o, "kernel_dW", lambda r, h, d: -orig_dw(r, h, d))
    with pytest.raises(AssertionError):
        test_linear_field_gradient_converges_to_the_exact_one()
    monkeypatch.setattr(o, "kernel_dW", orig_dw)
    # 2. the strong form with the pair sum instead of the difference
    monkeypatch.setattr(o, "gradients", lambda st, w, nb, prm: {
        **orig(st, w, nb, prm), "rho_strong": orig(st, w, nb, prm)["rho_weak"]})
    with pytest.raises(AssertionError):
        test_constant_field()
    # 3. m_j in place of V_j = m_j / rho_j (rho0 = 1000 makes it a factor of 1000)
    def mass_not_volume(st, w, nb, prm):
        s2 = st.copy()
        s2.m = st.m * st.rho
        return orig(s2, w, nb, prm)
    monkeypatch.setattr(o, "gradients", mass_not_volume)
    with pytest.raises(AssertionError):
        test_linear_field_gradient_converges_to_the_exact_one()
    # 4. the wall problem's extrapolation with the wrong sign of gravity
    def wrong_wall_sign(st, w, nb, prm):
        import copy
        p2 = copy.copy(prm)
        p2.gravity = -prm.gravity
        return orig(st, w, nb, p2)
    monkeypatch.setattr(o, "gradients", wrong_wall_sign)
    with pytest.raises(AssertionError):
        test_hydrostatic_pressure_gradient_reaches_the_walls()
    monkeypatch.setattr(o, "gradients", orig)
