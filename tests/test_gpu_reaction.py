"""GPU parity of the reaction step of reaction-diffusion (Eq. ode-spliting-2rd with the QSS
update of Eq. ode-qss; FitzHugh-Nagumo Eq. fhn and Aliev-Panfilov Eq. a-p) through the C ABI
against the FP64 oracle (oracle/reaction.py), and of diffusion and reaction alternated; and
the paper's spiral-wave test (a self-sustaining spiral against a planar wave that leaves).

Tolerance. The GPU holds V and w in FP32 and evaluates expf/expm1f in FP32: each of the four
reactions per step carries a few roundings of relative size 2^-24 on values of order 1, so
after k steps the difference stays below 1e-6 k (absolute), with margin for the mild
amplification of the excitable dynamics over the short runs used here.
"""
import numpy as np
import pytest

from oracle import diffusion as df
from oracle import reaction as rx
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.test_gpu_diffusion import _representable_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODELS = {
    "fn": dict(model=rx.FN, a=0.1, eps0=0.08, beta=1.0, gamma=1.0, sigma=0.02),
    "ap": dict(model=rx.AP, a=0.15, b=0.15, k=8.0, eps0=0.002, mu1=0.2, mu2=0.3),
}


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _setup(sph, n=40):
    prob = _representable_problem(wk.diffusion_band(n=n, ny=n, kappa=1e-3, a=0.2))
    sim = sph.Simulation(prob)
    sph.sph_build_cells(sim.handle)
    sp = sph.sph_species_create(sim.handle, prob.meta["D"][:2, :2], 2)
    return prob, sim, sp


@pytest.mark.parametrize("name", ["fn", "ap"])
def test_reaction_matches_oracle(sph, name):
    prob, sim, sp = _setup(sph)
    try:
        rng = np.random.default_rng(3)
        V0 = _f32(rng.uniform(0.0, 1.0, sim.n))
        w0 = _f32(rng.uniform(0.0, 0.3, sim.n))
        sph.sph_species_set(sim.handle, sp, V0)
        sph.sph_species_set_gate(sim.handle, sp, w0)
        r = sph.reaction_from(MODELS[name]["model"], **{k: v for k, v in MODELS[name].items() if k != "model"})
        steps, dt = 40, 0.02
        sph.sph_reaction_step(sim.handle, sp, r, dt, steps)
        Vg = sph.sph_species_get(sim.handle, sp, sim.n)
        wg = sph.sph_species_get_gate(sim.handle, sp, sim.n)
    finally:
        sph.sph_species_destroy(sp)
        sim.close()
    ro = rx.Reaction(**MODELS[name])
    V, w = V0.copy(), w0.copy()
    for _ in range(steps):
        V, w = rx.reaction_step(V, w, ro, dt)
    assert np.max(np.abs(V - V0)) > 1e-2                 # the system did evolve
    assert np.max(np.abs(Vg - V)) < 1e-6 * steps, np.max(np.abs(Vg - V))
    assert np.max(np.abs(wg - w)) < 1e-6 * steps, np.max(np.abs(wg - w))


def test_reaction_diffusion_alternated_matches_oracle(sph):
    # operator splitting of Sec. "SPH method for reaction-diffusion": a diffusion step and a
    # reaction step of the same dt, alternated, on the band of the first diffusion test
    prob, sim, sp = _setup(sph, n=48)
    name = "fn"
    try:
        V0 = _f32(prob.meta["C0"])
        sph.sph_species_set(sim.handle, sp, V0)
        r = sph.reaction_from(MODELS[name]["model"], **{k: v for k, v in MODELS[name].items() if k != "model"})
        dt = prob.meta["dt"]
        for _ in range(6):
            sph.sph_diffusion_step(sim.handle, sp, dt, 1)
            sph.sph_reaction_step(sim.handle, sp, r, dt, 1)
        Vg = sph.sph_species_get(sim.handle, sp, sim.n)
        wg = sph.sph_species_get_gate(sim.handle, sp, sim.n)
    finally:
        sph.sph_species_destroy(sp)
        sim.close()
    prm = o.Params.from_problem(prob)
    D = prob.meta["D"][:2, :2]
    V, w = V0.copy(), np.zeros_like(V0)
    ro = rx.Reaction(**MODELS[name])
    for _ in range(6):
        V = df.run(prob.pos, V, prob.mass, prob.rho, D, dt, 1, prm)
        V, w = rx.reaction_step(V, w, ro, dt)
    assert np.max(np.abs(Vg - V)) < 1e-5 and np.max(np.abs(wg - w)) < 1e-5


def _excite(sph, prob, T):
    """Aliev-Panfilov on the sheet: a diffusion step and a reaction step of dt, alternated, to
    time T; returns V at the end and the active fraction (V > 0.5) every 50 time units."""
    sim = sph.Simulation(prob)
    sph.sph_build_cells(sim.handle)
    sp = sph.sph_species_create(sim.handle, prob.meta["D"], 2)
    trace = []
    try:
        sph.sph_species_set(sim.handle, sp, prob.meta["C0"])
        sph.sph_species_set_gate(sim.handle, sp, prob.meta["w0"])
        r = sph.reaction_from(sph.SPH_REACTION_AP, **prob.meta["ap"])
        dt = prob.meta["dt"]
        per = int(round(50.0 / dt))
        for k in range(int(round(T / dt))):
            sph.sph_diffusion_step(sim.handle, sp, dt, 1)
            sph.sph_reaction_step(sim.handle, sp, r, dt, 1)
            if (k + 1) % per == 0:
                trace.append(float(np.mean(sph.sph_species_get(sim.handle, sp, sim.n) > 0.5)))
        V = sph.sph_species_get(sim.handle, sp, sim.n)
    finally:
        sph.sph_species_destroy(sp)
        sim.close()
    return V, trace


def test_spiral_wave_sustains_itself_and_a_planar_wave_leaves(sph):
    # the paper's spiral-wave test in the Aliev-Panfilov model's units: from a cross-field
    # start (excited lower-left quarter, refractory upper-left quarter) the front's free end
    # curls into a spiral that keeps a steady share of the sheet excited, while a planar wave
    # started at the left edge crosses the sheet and leaves it at rest
    T = 300.0
    V_spiral, tr_spiral = _excite(sph, wk.excitable_sheet(200, 0.5, cross_field=True), T)
    V_plane, tr_plane = _excite(sph, wk.excitable_sheet(200, 0.5, cross_field=False), T)
    print("active fraction every 50 units, spiral:", [f"{a:.3f}" for a in tr_spiral],
          "planar:", [f"{a:.3f}" for a in tr_plane])
    assert np.all(np.isfinite(V_spiral)) and np.all(np.isfinite(V_plane))
    assert min(tr_spiral[1:]) > 0.1 and max(tr_spiral) < 0.6
    assert tr_plane[-1] < 0.01 and max(tr_plane) > 0.05


def test_reaction_edge_cases(sph):
    prob, sim, sp = _setup(sph, n=16)
    try:
        w0 = _f32(np.linspace(0.0, 0.5, sim.n))
        sph.sph_species_set_gate(sim.handle, sp, w0)
        assert np.array_equal(sph.sph_species_get_gate(sim.handle, sp, sim.n), w0)
        r = sph.reaction_from(sph.SPH_REACTION_FN, a=0.1, eps0=0.08, beta=1.0, gamma=1.0)
        sph.sph_reaction_step(sim.handle, sp, r, 0.1, 0)                 # zero steps: no change
        assert np.array_equal(sph.sph_species_get_gate(sim.handle, sp, sim.n), w0)
        for bad_dt in (0.0, -0.1, float("nan")):
            with pytest.raises(sph.SphError):
                sph.sph_reaction_step(sim.handle, sp, r, bad_dt, 1)
        with pytest.raises(sph.SphError):
            sph.sph_reaction_step(sim.handle, sp, sph.reaction_from(7, a=0.1), 0.1, 1)
        with pytest.raises(sph.SphError):
            sph.sph_reaction_step(sim.handle, sp, sph.reaction_from(sph.SPH_REACTION_FN, a=float("inf")), 0.1, 1)
        # the rest state of both models is a fixed point, bit for bit
        sph.sph_species_set(sim.handle, sp, np.zeros(sim.n))
        sph.sph_species_set_gate(sim.handle, sp, np.zeros(sim.n))
        sph.sph_reaction_step(sim.handle, sp, r, 0.1, 10)
        ap = sph.reaction_from(sph.SPH_REACTION_AP, a=0.15, b=0.15, k=8.0, eps0=0.002, mu1=0.2, mu2=0.3)
        sph.sph_reaction_step(sim.handle, sp, ap, 0.1, 10)
        assert np.all(sph.sph_species_get(sim.handle, sp, sim.n) == 0.0)
        assert np.all(sph.sph_species_get_gate(sim.handle, sp, sim.n) == 0.0)
    finally:
        sph.sph_species_destroy(sp)
        sim.close()
