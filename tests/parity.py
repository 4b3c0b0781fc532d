"""Shared helpers of the GPU parity tests: representable states and error norms.

The GPU holds positions as fixed-point integers, velocities and d rho/dt in
FP32 and rho - rho0 in FP32 (see include/sph.h). Parity cases hand both sides
the same state, already rounded to that representation, so any difference
comes from the arithmetic and not from the input.
"""
import numpy as np

from oracle import wcsph as o

REL_L2_TOL = 1e-5            # per-substep tolerance on rho, dv/dt and v (relative L2)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def representable(problem, x, v, rho, drho=None):
    """Round a state to what the GPU stores exactly, using the oracle's own reading
    of the position contract."""
    prm = o.Params.from_problem(problem)
    xq = o.dequantise(o.quantise(np.asarray(x, dtype=np.float64), prm), prm)
    v32 = np.asarray(v, dtype=np.float32).astype(np.float64)
    dev = (np.asarray(rho, dtype=np.float64) - prm.rho0).astype(np.float32).astype(np.float64)
    rho32 = prm.rho0 + dev
    d32 = None if drho is None else np.asarray(drho, dtype=np.float32).astype(np.float64)
    return xq, v32, rho32, d32


def walls_representable(problem):
    prm = o.Params.from_problem(problem)
    w = np.asarray(problem.wall_pos, dtype=np.float64)
    if w.size == 0:
        return w
    return o.dequantise(o.quantise(w, prm), prm)


def perturbed_state(problem, seed, vel_amp, rho_amp):
    """Seeded random velocity / density perturbation of a problem's initial state."""
    rng = np.random.default_rng(seed)
    x = np.asarray(problem.pos, dtype=np.float64)
    v = np.asarray(problem.vel, dtype=np.float64) + rng.uniform(-vel_amp, vel_amp, size=x.shape)
    rho = np.asarray(problem.rho, dtype=np.float64) * (1.0 + rng.uniform(0, rho_amp, size=x.shape[0]))
    drho = rng.uniform(-rho_amp, rho_amp, size=x.shape[0])
    return x, v, rho, drho
