"""Training and use of the learned stand-in for the acoustic substeps.

The network (definition in include/sph.h, sph_learned_*) runs entirely in libsph.so:
forward, backward and Adam are the library's kernels. This module only orchestrates:
it runs the plain solver to record training pairs (the state at the start of an
advection step, after density re-initialisation, and the state at its end), feeds them
to sph_learned_train_step, and compares learned stepping against plain stepping.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import sph, workloads

ORDER = ("enc", "e1", "e2", "n1", "n2", "d1", "d2")
SHAPES = {"enc": (64, 16), "e1": (64, 80), "e2": (64, 80), "n1": (64, 144), "n2": (64, 80),
          "d1": (64, 80), "d2": (16, 80)}
S_RHO = 100.0


def initial_weights(dim: int, seed: int = 0) -> np.ndarray:
    """He-normal weights on the live input columns of each matrix (biases and padding 0),
    the last layer of each residual / output branch scaled by 0.1."""
    rng = np.random.default_rng(seed)
    fan = {"enc": dim + 3, "e1": 2 * dim + 3 + 64 + 1, "e2": 65, "n1": 129, "n2": 65, "d1": 65, "d2": 65}
    parts = []
    for name in ORDER:
        r, c = SHAPES[name]
        w = np.zeros((r, c), dtype=np.float32)
        k = fan[name]
        w[:, :k - 1] = rng.normal(0.0, math.sqrt(2.0 / k), size=(r, k - 1))
        if name in ("e2", "n2", "d2"):
            w *= 0.1
        if name == "d2":
            w[dim + 1:, :] = 0.0
        parts.append(w.ravel())
    return np.concatenate(parts)


@dataclass
class Sample:
    tank: int
    pos: np.ndarray
    vel: np.ndarray
    rho: np.ndarray
    drho: np.ndarray
    t: float
    target: np.ndarray


@dataclass
class Dataset:
    problems: list
    samples: list = field(default_factory=list)


def targets(problem, vel0, vel1, rho0_arr, rho1_arr, dt_ad):
    """[(dv - g dt_ad)/V_S, 100 drho/rho0] with V_S = |g| dt_ad (U_ref without gravity)."""
    d = problem.dim
    g = np.asarray(problem.gravity, dtype=np.float64)[:d]
    vs = float(np.linalg.norm(g)) * dt_ad or problem.u_ref
    T = np.empty((vel0.shape[0], d + 1))
    T[:, :d] = (vel1 - vel0 - g * dt_ad) / vs
    T[:, d] = S_RHO * (rho1_arr - rho0_arr) / problem.rho0
    return T


def training_tanks(n_tanks=200, n_per_H=40, base_seed=workloads.BATCH_BASE_SEED):
    """Seeded dam-break geometries: H ~ U(0.5, 1.5), L/H ~ U(1, 3), dp = H / n_per_H."""
    out = []
    for s in range(n_tanks):
        u = workloads._uniforms(base_seed ^ (0x5EED0000 + s), 2)
        H = 0.5 + u[0]
        L = H * (1.0 + 2.0 * u[1])
        out.append(workloads.dam_break(dim=2, H=H, L=L, dp=H / n_per_H, name=f"train_{s}"))
    return out


def record(problems, steps=300, every=15, stream=None) -> Dataset:
    """Run the plain GPU solver on each tank and keep every `every`-th advection step as a
    (start state, target) pair."""
    data = Dataset(problems=problems)
    for k, p in enumerate(problems):
        sim = sph.Simulation(p, stream=stream)
        for step in range(steps):
            sim.build_cells()
            dt_ad = sim.advection_step()
            keep = step % every == every // 2
            if keep:
                pos, vel, rho, drho = sim.state()
                t0 = sim.diagnostics()["t"]
            while not sim.acoustic_substep()[0]:
                pass
            if keep:
                _, vel1, rho1, _ = sim.state()
                data.samples.append(Sample(k, pos, vel, rho, drho, t0,
                                           targets(p, vel, vel1, rho, rho1, dt_ad)))
        sim.close()
    return data


def train(net, data: Dataset, epochs=4, lr=1e-3, lr_final=1e-4, seed=0, stream=None, log=None):
    """Adam on the recorded pairs, one sample per step, shuffled each epoch, with a
    geometric learning-rate decay. Returns the loss history."""
    sims = {}
    rng = np.random.default_rng(seed)
    losses = []
    total = epochs * len(data.samples)
    it = 0
    for ep in range(epochs):
        for idx in rng.permutation(len(data.samples)):
            s = data.samples[idx]
            sim = sims.get(s.tank)
            if sim is None:
                sim = sims[s.tank] = sph.Simulation(data.problems[s.tank], stream=stream)
            sim.set_state(s.pos, s.vel, s.rho, s.drho, t=s.t)
            sim.build_cells()
            sim.advection_step()
            rate = lr * (lr_final / lr) ** (it / max(total - 1, 1))
            loss, _ = sph.sph_learned_train_step(sim.handle, net, s.target, rate, stream=stream)
            losses.append(loss)
            it += 1
        if log:
            log(f"epoch {ep}: mean loss {np.mean(losses[-len(data.samples):]):.4g}")
    for sim in sims.values():
        sim.close()
    return losses


def evaluation_loss(net, data: Dataset, stream=None):
    """Mean loss of the network on recorded pairs (no update)."""
    sims, out = {}, []
    for s in data.samples:
        sim = sims.get(s.tank)
        if sim is None:
            sim = sims[s.tank] = sph.Simulation(data.problems[s.tank], stream=stream)
        sim.set_state(s.pos, s.vel, s.rho, s.drho, t=s.t)
        sim.build_cells()
        sim.advection_step()
        loss, _ = sph.sph_learned_train_step(sim.handle, net, s.target, 0.0, stream=stream)
        out.append(loss)
    for sim in sims.values():
        sim.close()
    return float(np.mean(out))


def compare_stepping(net, problem, steps, max_mean_rho_dev=0.01, max_energy_drift=0.005, stream=None):
    """Learned stepping (with its fallback) against plain stepping from the same start.
    Returns wall times per advection step, the fraction of learned steps kept and the
    relative energy difference of the two runs at the end."""
    import torch
    plain = sph.Simulation(problem, flags=sph.SPH_FLAG_GRAPH, stream=stream)
    learn = sph.Simulation(problem, stream=stream)
    plain.step(1)
    learn.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain.step(steps)
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / steps
    kept = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        kept += sph.sph_learned_step(learn.handle, net, max_mean_rho_dev, max_energy_drift, stream=stream)
    torch.cuda.synchronize()
    t_learn = (time.perf_counter() - t0) / steps
    dp, dl = plain.diagnostics(), learn.diagnostics()
    e0 = abs(dp["energy"])
    out = {"plain_ms_per_step": 1e3 * t_plain, "learned_ms_per_step": 1e3 * t_learn,
           "speedup": t_plain / t_learn, "kept_fraction": kept / steps,
           "energy_rel_diff": abs(dl["energy"] - dp["energy"]) / e0,
           "t_plain": dp["t"], "t_learned": dl["t"],
           "front_plain": dp["front_x"], "front_learned": dl["front_x"]}
    plain.close()
    learn.close()
    return out
