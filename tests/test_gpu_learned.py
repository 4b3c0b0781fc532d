"""The learned stand-in on the GPU against its FP64 reference (oracle/mpnn.py): forward
outputs, hand-written gradients, training, and the learned advection step with fallback."""
import copy

import numpy as np
import pytest

from oracle import mpnn
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import perturbed_state, rel_l2, representable, walls_representable

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = ["enc", "e1", "e2", "n1", "n2", "d1", "d2"]


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def pack(W):
    return np.concatenate([W[k].ravel() for k in ORDER]).astype(np.float32)


def unpack(flat, dim):
    out, o_ = {}, 0
    for k in ORDER:
        r, c = mpnn.layer_shapes(dim)[k]
        out[k] = flat[o_:o_ + r * c].reshape(r, c).astype(np.float64)
        o_ += r * c
    return out


def _case(dim, seed=0):
    if dim == 2:
        prob = wk.dam_break(dim=2, H=0.3, L=0.4, dp=0.02, tank=1.0)
    else:
        prob = wk.dam_break(dim=3, H=0.2, L=0.25, W=0.2, dp=0.025, tank=0.6)
    prob.wall_pos = walls_representable(prob)
    x, v, rho, drho = perturbed_state(prob, seed, 0.3, 0.01)
    x = x + np.random.default_rng(seed + 1).uniform(-0.1, 0.1, x.shape) * prob.dp
    return prob, representable(prob, x, v, rho, drho)


def _start_of_step(sph, prob, state):
    """Handle at the start of an advection step (cells built, density re-initialised)."""
    sim = sph.Simulation(prob)
    sim.set_state(*state, t=0.0)
    sim.build_cells()
    dt_ad = sim.advection_step()
    pos, vel, rho, _ = sim.state()
    return sim, dt_ad, pos, vel, rho


def _oracle_graph(prob, pos, vel, rho, dt_ad):
    prm = o.Params.from_problem(prob)
    I, J, IW, KW = o.neighbour_sets_quantised(pos, prob.wall_pos, prm)
    return mpnn.build_graph(prob.dim, pos, vel, rho, prob.wall_pos, I, J, IW, KW, prob.h, prob.c0,
                            prob.rho0, dt_ad)


@pytest.mark.parametrize("dim", [2, 3])
def test_forward_matches_reference(sph, dim):
    prob, state = _case(dim)
    W = mpnn.init_weights(dim, seed=5)
    net = sph.sph_learned_create(dim, pack(W))
    sim, dt_ad, pos, vel, rho = _start_of_step(sph, prob, state)
    y = sph.sph_learned_predict(sim.handle, net, prob.n_fluid, dim)
    g = _oracle_graph(prob, pos, vel, rho, dt_ad)
    Y, _ = mpnn.forward(unpack(pack(W), dim), g)
    err = rel_l2(y, Y)
    print(f"{dim}D forward: rel L2 {err:.2e} over {y.size} outputs, {g.src.size} edges")
    assert err < 2e-3
    sph.sph_learned_destroy(net)
    sim.close()


FUSED_FORMS = [1, 2]     # warp-level MMA rounds; tcgen05 pipeline


@pytest.mark.parametrize("form", FUSED_FORMS)
@pytest.mark.parametrize("dim", [2, 3])
def test_fused_inference_equals_the_unfused_layers(sph, dim, form):
    # the fused edge rounds make the same products, roundings and sums in the same order
    prob, state = _case(dim, seed=2)
    net = sph.sph_learned_create(dim, pack(mpnn.init_weights(dim, seed=6)))
    sph.sph_learned_set_fused(net, form)
    sim, _, _, _, _ = _start_of_step(sph, prob, state)
    y_fused = sph.sph_learned_predict(sim.handle, net, prob.n_fluid, dim)
    sph.sph_learned_set_fused(net, False)
    y_plain = sph.sph_learned_predict(sim.handle, net, prob.n_fluid, dim)
    assert np.abs(y_plain).max() > 0
    np.testing.assert_array_equal(y_fused, y_plain)
    sph.sph_learned_destroy(net)
    sim.close()


def test_all_forms_agree_bit_for_bit_at_100k_particles(sph):
    # 2M edges: every dense-layer CTA walks several 128-row tiles (both tile buffers), and the
    # fused kernels run many node runs per CTA; the three forms must agree exactly
    from paper_2010_12375_gb300 import learned
    prob = wk.learned_dam_break()
    sim = sph.Simulation(prob, flags=sph.SPH_FLAG_GRAPH)
    sim.step(2)
    sim.build_cells()
    sim.advection_step()
    net = sph.sph_learned_create(2, learned.initial_weights(2, seed=0))
    ys = []
    for form in (0, 1, 2):
        sph.sph_learned_set_fused(net, form)
        ys.append(sph.sph_learned_predict(sim.handle, net, prob.n_fluid, 2))
    assert np.all(np.isfinite(ys[0])) and np.abs(ys[0]).max() > 0
    np.testing.assert_array_equal(ys[1], ys[0])
    np.testing.assert_array_equal(ys[2], ys[0])
    sph.sph_learned_destroy(net)
    sim.close()


def test_fused_form_outside_the_range_is_rejected(sph):
    net = sph.sph_learned_create(2, pack(mpnn.init_weights(2, seed=1)))
    for bad in (-1, 3):
        with pytest.raises(sph.SphError):
            sph.sph_learned_set_fused(net, bad)
    sph.sph_learned_destroy(net)


@pytest.mark.parametrize("form", FUSED_FORMS)
def test_fused_inference_with_edgeless_nodes(sph, form):
    # five particles lifted into the empty upper tank, > 2h from everything: nodes without
    # edges between nodes with edges, in the fused kernel's node runs and edge tiles
    prob, (x, v, rho, drho) = _case(2, seed=4)
    x = x.copy()
    for k in range(5):
        x[7 * k + 3] = (0.1 + 0.15 * k, 0.8)
    state = representable(prob, x, v, rho, drho)
    net = sph.sph_learned_create(2, pack(mpnn.init_weights(2, seed=8)))
    sph.sph_learned_set_fused(net, form)
    sim, _, _, _, _ = _start_of_step(sph, prob, state)
    fc, wc, _, _ = sim.neighbours()
    assert np.count_nonzero(fc + wc == 0) >= 5
    y_fused = sph.sph_learned_predict(sim.handle, net, prob.n_fluid, 2)
    sph.sph_learned_set_fused(net, False)
    y_plain = sph.sph_learned_predict(sim.handle, net, prob.n_fluid, 2)
    np.testing.assert_array_equal(y_fused, y_plain)
    sph.sph_learned_destroy(net)
    sim.close()


@pytest.mark.parametrize("form", FUSED_FORMS)
def test_fused_inference_single_particle(sph, form):
    # no edges at all: every round's messages are zero
    prob = wk.dam_break(dim=2, H=0.3, L=0.4, dp=0.02, tank=1.0)
    prob.wall_pos = walls_representable(prob)
    single = copy.copy(prob)
    single.pos = np.array([[0.5, 0.5]])
    single.vel = np.array([[0.1, -0.2]])
    single.rho = np.array([prob.rho0])
    single.mass = prob.mass[:1]
    net = sph.sph_learned_create(2, pack(mpnn.init_weights(2, seed=9)))
    sph.sph_learned_set_fused(net, form)
    sim = sph.Simulation(single)
    sim.build_cells()
    sim.advection_step()
    y_fused = sph.sph_learned_predict(sim.handle, net, 1, 2)
    sph.sph_learned_set_fused(net, False)
    y_plain = sph.sph_learned_predict(sim.handle, net, 1, 2)
    assert np.all(np.isfinite(y_fused))
    np.testing.assert_array_equal(y_fused, y_plain)
    sph.sph_learned_destroy(net)
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_gradients_match_reference(sph, dim):
    prob, state = _case(dim, seed=3)
    W = mpnn.init_weights(dim, seed=7)
    net = sph.sph_learned_create(dim, pack(W))
    sim, dt_ad, pos, vel, rho = _start_of_step(sph, prob, state)
    T = np.random.default_rng(9).normal(0, 1.0, (prob.n_fluid, dim + 1))
    loss, grad = sph.sph_learned_train_step(sim.handle, net, T, 0.0, want_grad=True)
    g = _oracle_graph(prob, pos, vel, rho, dt_ad)
    Wd = unpack(pack(W), dim)
    Y, cache = mpnn.forward(Wd, g)
    dW = mpnn.backward(Wd, g, cache, Y, T)
    assert abs(loss - mpnn.loss(Y, T)) < 1e-3 * mpnn.loss(Y, T)
    gw = unpack(grad, dim)
    for k in ORDER:
        err = rel_l2(gw[k], dW[k])
        print(f"{dim}D grad {k}: rel L2 {err:.2e}")
        assert err < 1e-3, (k, err)
    sph.sph_learned_destroy(net)
    sim.close()


def test_adam_step_and_training(sph):
    prob, state = _case(2, seed=4)
    W0 = pack(mpnn.init_weights(2, seed=1))
    net = sph.sph_learned_create(2, W0)
    sim, dt_ad, pos, vel, rho = _start_of_step(sph, prob, state)
    T = np.random.default_rng(2).normal(0, 0.5, (prob.n_fluid, 3))
    lr = 3e-3
    # the first Adam step from zero moments, applied to the gradient the GPU computes
    _, grad = sph.sph_learned_train_step(sim.handle, net, T, 0.0, want_grad=True)
    m = 0.1 * grad.astype(np.float64)
    v = 0.001 * grad.astype(np.float64) ** 2
    expect = -lr * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    loss0, _ = sph.sph_learned_train_step(sim.handle, net, T, lr)
    got = sph.sph_learned_get_weights(net).astype(np.float64) - W0
    assert rel_l2(got, expect) < 1e-5
    losses = [loss0] + [sph.sph_learned_train_step(sim.handle, net, T, lr)[0] for _ in range(79)]
    assert losses[-1] < 0.85 * losses[0]
    assert np.all(np.isfinite(sph.sph_learned_get_weights(net)))
    sph.sph_learned_destroy(net)
    sim.close()


def test_rejected_learned_step_falls_back_to_the_plain_step(sph):
    prob = wk.dam_break_2d(n_per_H=20)
    W = mpnn.init_weights(2, seed=0)
    W["d2"][2, -1] = 0.0
    W["d2"][2, 64] = 50.0           # bias of the density output: +0.5 rho0 per step, far past 1 %
    net = sph.sph_learned_create(2, pack(W))
    a = sph.Simulation(prob)
    b = sph.Simulation(prob)
    a.step(3)
    b.step(3)
    used = sph.sph_learned_step(a.handle, net, 0.01, 0.005)
    assert not used
    b.step(1)
    for u, v in zip(a.state(), b.state()):
        np.testing.assert_array_equal(u, v)
    da, db = a.diagnostics(), b.diagnostics()
    assert da["t"] == db["t"] and da["substeps"] == db["substeps"]
    sph.sph_learned_destroy(net)
    a.close()
    b.close()


def test_accepted_learned_step_advances_the_clock(sph):
    prob = wk.dam_break_2d(n_per_H=20)
    net = sph.sph_learned_create(2, np.zeros(sph.sph_learned_weight_count(), dtype=np.float32))
    sim = sph.Simulation(prob)
    d0 = sim.diagnostics()
    used = sph.sph_learned_step(sim.handle, net, 0.01, 0.005)
    d1 = sim.diagnostics()
    # zero weights predict pure gravity over the step: free fall conserves energy
    assert used
    assert d1["t"] > d0["t"] and d1["substeps"] == d0["substeps"]
    pos, vel, rho, _ = sim.state()
    np.testing.assert_allclose(vel[:, 1], -d1["t"], rtol=1e-5)
    sph.sph_learned_destroy(net)
    sim.close()


def test_trained_network_gains_over_the_untrained_predictor(sph):
    """Trained on recorded solver steps, the network predicts held-out steps much better
    than the gravity-only prediction (zero network); the learned stepping's cost against
    the plain substeps is measured and printed."""
    from paper_2010_12375_gb300 import learned
    tanks = learned.training_tanks(n_tanks=24, n_per_H=20)
    data = learned.record(tanks[:20], steps=90, every=15)
    held = learned.record(tanks[20:], steps=90, every=15)
    net = sph.sph_learned_create(2, learned.initial_weights(2, seed=0))
    zero = sph.sph_learned_create(2, np.zeros(sph.sph_learned_weight_count(), dtype=np.float32))
    base = learned.evaluation_loss(zero, held)
    learned.train(net, data, epochs=6, lr=2e-3, lr_final=2e-4)
    after = learned.evaluation_loss(net, held)
    print(f"held-out loss: gravity-only {base:.4g}, trained {after:.4g}")
    assert after < 0.5 * base
    cmp = learned.compare_stepping(net, wk.dam_break_2d(n_per_H=20), steps=20)
    print("learned vs plain stepping:", cmp)
    assert cmp["kept_fraction"] >= 0.0 and cmp["plain_ms_per_step"] > 0
    sph.sph_learned_destroy(net)
    sph.sph_learned_destroy(zero)


def test_training_steps_are_bit_reproducible(sph):
    # every reduction of forward, backward and Adam runs in a fixed order
    prob, state = _case(2, seed=6)
    W0 = pack(mpnn.init_weights(2, seed=2))
    a = sph.sph_learned_create(2, W0)
    b = sph.sph_learned_create(2, W0)
    sim, dt_ad, pos, vel, rho = _start_of_step(sph, prob, state)
    T = np.random.default_rng(3).normal(0, 0.5, (prob.n_fluid, 3))
    for _ in range(3):
        sph.sph_learned_train_step(sim.handle, a, T, 2e-3)
        sph.sph_learned_train_step(sim.handle, b, T, 2e-3)
    wa, wb = sph.sph_learned_get_weights(a), sph.sph_learned_get_weights(b)
    assert np.any(wa != W0)
    np.testing.assert_array_equal(wa, wb)
    sph.sph_learned_destroy(a)
    sph.sph_learned_destroy(b)
    sim.close()
