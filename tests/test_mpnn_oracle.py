"""Pins of the learned stand-in's FP64 reference: the hand-written backward pass against
central finite differences, and the bfloat16 rounding against its definition."""
import numpy as np
import pytest

from oracle import mpnn
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk


def _tiny_graph(dim=2, seed=0):
    prob = wk.dam_break(dim=dim, H=0.2, L=0.2, dp=0.05, tank=0.4) if dim == 2 else \
        wk.dam_break(dim=3, H=0.15, L=0.15, W=0.15, dp=0.05, tank=0.3)
    rng = np.random.default_rng(seed)
    prm = o.Params.from_problem(prob)
    x = prob.pos + rng.uniform(-0.1, 0.1, prob.pos.shape) * prob.dp
    v = rng.uniform(-0.3, 0.3, prob.pos.shape)
    rho = 1.0 + rng.uniform(0, 0.01, prob.n_fluid)
    I, J, IW, KW = o.neighbour_sets(x, prob.wall_pos, prm)
    g = mpnn.build_graph(dim, x, v, rho, prob.wall_pos, I, J, IW, KW, prob.h, prob.c0, 1.0, 0.01)
    T = rng.normal(0, 0.5, (prob.n_fluid, dim + 1))
    return g, T


def test_bf16_rounding_matches_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.3, 1e-3, 0.0])
    r = mpnn.bf16(x)
    assert r[0] == 1.0 and r[-1] == 0.0
    # ties go to even: 1 + 2^-8 lies between 1 and 1 + 2^-7 -> 1 (even mantissa)
    assert mpnn.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mpnn.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    m = np.frexp(np.abs(r[np.abs(r) > 0]))[0]
    assert np.all(np.abs(m * 256 - np.round(m * 256)) < 1e-12)      # 8 significant bits
    assert np.max(np.abs(r - x) / np.maximum(np.abs(x), 1e-300)) <= 2 ** -8   # half an ulp


@pytest.mark.parametrize("dim", [2, 3])
def test_backward_matches_finite_differences(dim):
    g, T = _tiny_graph(dim)
    W = mpnn.init_weights(dim, seed=3)
    for k in W:                                     # make every layer matter
        W[k] = W[k] + 0.05 * np.random.default_rng(7).normal(size=W[k].shape) * (W[k] != 0)
    Y, cache = mpnn.forward(W, g, q=False)
    dW = mpnn.backward(W, g, cache, Y, T, q=False)
    rng = np.random.default_rng(11)
    eps = 1e-6
    for name in W:
        rows, cols = np.nonzero(W[name])
        pick = rng.choice(rows.size, size=min(6, rows.size), replace=False)
        for p in pick:
            r, c = rows[p], cols[p]
            Wp = {k: v.copy() for k, v in W.items()}
            Wm = {k: v.copy() for k, v in W.items()}
            Wp[name][r, c] += eps
            Wm[name][r, c] -= eps
            fd = (mpnn.loss(mpnn.forward(Wp, g, q=False)[0], T) -
                  mpnn.loss(mpnn.forward(Wm, g, q=False)[0], T)) / (2 * eps)
            assert abs(fd - dW[name][r, c]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (name, r, c, fd, dW[name][r, c])


def test_planted_backward_mistake_is_caught(monkeypatch):
    g, T = _tiny_graph(2)
    W = mpnn.init_weights(2, seed=3)
    orig = mpnn.nbar
    Y, cache = mpnn.forward(W, g, q=False)
    monkeypatch.setattr(mpnn, "nbar", lambda d: 2 * orig(d))    # backward forgets a factor
    dW = mpnn.backward(W, g, cache, Y, T, q=False)
    monkeypatch.setattr(mpnn, "nbar", orig)
    eps = 1e-6
    Wp = {k: v.copy() for k, v in W.items()}
    Wm = {k: v.copy() for k, v in W.items()}
    Wp["e1"][0, 0] += eps
    Wm["e1"][0, 0] -= eps
    fd = (mpnn.loss(mpnn.forward(Wp, g, q=False)[0], T) - mpnn.loss(mpnn.forward(Wm, g, q=False)[0], T)) / (2 * eps)
    assert abs(fd - dW["e1"][0, 0]) > 1e-4 * abs(fd)


def test_training_reduces_the_loss():
    g, T = _tiny_graph(2, seed=1)
    W = mpnn.init_weights(2, seed=0)
    m = {k: np.zeros_like(v) for k, v in W.items()}
    v = {k: np.zeros_like(w) for k, w in W.items()}
    opt = mpnn.Adam(lr=3e-3)
    first = None
    for t in range(1, 61):
        Y, cache = mpnn.forward(W, g)
        L = mpnn.loss(Y, T)
        first = first if first is not None else L
        mpnn.adam_step(W, mpnn.backward(W, g, cache, Y, T), m, v, t, opt)
    assert L < 0.5 * first
