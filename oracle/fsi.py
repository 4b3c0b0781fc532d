"""Plain FP64 CPU oracle of the multi-resolution fluid-structure coupling (test
infrastructure only: only the tests, the smoke check and the benchmark's CPU legs may use
it; it shares no code with the CUDA library).

The method, in the paper's order:
  * Total Lagrangian solid (Sec. "Total Lagrangian formulation"): neighbours fixed in the
    reference configuration; correction matrix B0 (Eq. sph-correctmatrix); deformation
    gradient F; first Piola-Kirchhoff stress P = F S from the linear-elastic law
    (Eq. isotropic-linear-elasticity) or the Neo-Hookean energy (S = dW/dE); momentum
    (Eq. sph-mechanical-mom) with the inter-particle average P~_ab = (P_a B0_a + P_b B0_b)/2.
  * Solid position-based Verlet (Eqs. verlet-first-half-solid, verlet-first-mediate-solid,
    verlet-first-final-solid) with the solid time step of Eq. dts-advection.
  * Multi-resolution coupling (Sec. "Multi-resolution FSI coupling"): the fluid sees the
    solid particles through the fluid kernel W(r, h_F) with the imaginary pressure and
    velocity of Eq. fs-coupling-mr; the pressure force Eq. fs-force-mr-sp and the viscous
    force Eq. fs-force-mr-sv act on the fluid, their reactions on the solid; per fluid
    acoustic step, kappa = [dt_F / dt_S] + 1 solid steps.

Readings (the same the CUDA path takes):
  R2  (as in wcsph) the kernel gradient is the true gradient grad_a W_ab = dW/dr r_ab/|r_ab|,
      r_ab = r_a - r_b. With it B0 is close to +I on a lattice, F = I + grad u exactly for a
      linear displacement, and 2 sum V_b P~ grad W / rho0 is div P^T (the paper's own sign
      convention flips B0 as well, which gives the same F and the same forces).
  R19 E = 2G(1 + nu) = 3K(1 - 2nu) (the printed 2G(1 + 2nu) is read as the standard
      relation); K = lambda + 2mu/3 as printed; c_S = sqrt(K / rho0_S).
  R20 dF/dt is evaluated in the second half of a solid step from the new velocities
      (dF/dt = (sum_b V_b (v_b - v_a) (x) grad0 W_ab) B0_a) and carried into the first half of
      the next one (zero at the start), as d rho/dt is for the fluid.
  R21 f^{S:p}, f^{S:v} (Eqs. fs-force-mr-sp, fs-force-mr-sv) are forces: they enter the fluid's
      dv/dt divided by m_i, and their reactions enter the solid's divided by m_a.
  R22 imaginary pressure p_a^d = p_i + rho_i max(0, -(g - a~_a).n_a) ((r_i - r_a).n_a), n_a the
      solid's unit normal pointing into the fluid. For a solid at rest under gravity this is
      the hydrostatic extrapolation p_i + rho_i g (depth difference), the wall problem's P_R
      (Eq. eqriepright); the printed orientation of n and r_ia gives no extrapolation either
      way round, so it is read this way. rho_a^d from the EoS.
  R23 imaginary velocity v_a^d = 2 v~_a - v_i (the no-slip mirror about the solid's velocity);
      the printed 2 v_i - v~_a would make the viscous force anti-diffusive with dW/dr < 0.
  R24 the fluid's pressure and viscous forces on the solid are evaluated once per fluid
      acoustic step, in its pressure relaxation, and held over that step's kappa solid steps;
      v~_a and a~_a are the solid's velocity and acceleration averaged over the previous fluid
      step's solid steps (zero at the start).
  R25 the kappa solid steps of a fluid step have equal length dt_F / kappa, so that they cover
      the fluid step; dt_S is evaluated at the start of the fluid step.
  R26 order of a fluid acoustic step: fluid pressure relaxation (fluid, walls, solid at its
      current positions, fluid at the mid point), fluid density relaxation (the solid as a
      moving wall in the continuity equation, fluid at the new positions), then the solid's
      kappa steps.
  R27 every solid particle carries the unit normal of the wetted surface nearest to it, in
      the reference configuration (not rotated: small deformations).
  R28 in the continuity equation a solid neighbour is a moving wall (Eqs. eqriepartial,
      eqrienoslip with the wall velocity u_w = -n_a.v~_a): U_L = -n_a.v_i, U_R = -U_L + 2 u_w,
      P_L = p_i, P_R = p_a^d, rho_R from the EoS, and the term 2 rho_i V_a (U* - U_L) dW/dr.
  R29 clamped (fixed) solid particles keep their reference position and zero velocity; they
      take part in the stress and F like the others.
  R30 solid particles take no part in the fluid's density re-initialisation (Eq. eqrhosum):
      fluid next to the solid keeps its continuity density through the free-surface max.

Parity pins: tests/test_fsi_oracle.py (closed forms, invariants, brute force, planted
mistakes). None is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

from oracle import wcsph as o

LINEAR, NEO_HOOKEAN = 1, 2


@dataclass
class Material:
    rho0: float
    youngs: float
    poisson: float
    model: int = LINEAR

    @property
    def mu(self) -> float:                       # shear modulus G (R19)
        return self.youngs / (2.0 * (1.0 + self.poisson))

    @property
    def lam(self) -> float:
        nu = self.poisson
        return self.youngs * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))

    @property
    def K(self) -> float:                        # K = lambda + 2 mu / 3 as printed
        return self.lam + 2.0 * self.mu / 3.0

    @property
    def c(self) -> float:                        # c_S = sqrt(K / rho0)
        return math.sqrt(self.K / self.rho0)


@dataclass
class Solid:
    x0: np.ndarray            # (Ns, d) reference positions
    x: np.ndarray             # (Ns, d) current positions
    v: np.ndarray             # (Ns, d)
    F: np.ndarray             # (Ns, d, d) deformation gradient
    dFdt: np.ndarray          # (Ns, d, d) carried from the last second half (R20)
    V: np.ndarray             # (Ns,) reference volumes
    n: np.ndarray             # (Ns, d) unit normals into the fluid (R27)
    fixed: np.ndarray         # (Ns,) bool, clamped (R29)
    B0: np.ndarray            # (Ns, d, d)
    I: np.ndarray             # reference neighbour pairs (directed, both orders)
    J: np.ndarray
    gW: np.ndarray            # (pairs, d) grad0_a W_ab at the reference configuration
    mat: Material
    h: float
    gravity: np.ndarray
    acc: np.ndarray = None    # last dv/dt
    vbar: np.ndarray = None   # v~ over the last fluid step (R24)
    abar: np.ndarray = None   # a~ over the last fluid step
    f_fluid: np.ndarray = None  # fluid force held over the solid steps (R24)

    @property
    def m(self) -> np.ndarray:
        return self.mat.rho0 * self.V

    def copy(self) -> "Solid":
        c = Solid(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in self.__dict__.items()})
        return c


def _scatter(idx, vals, n):
    if vals.ndim == 1:
        return np.bincount(idx, weights=vals, minlength=n)
    flat = vals.reshape(vals.shape[0], -1)
    out = np.stack([np.bincount(idx, weights=flat[:, k], minlength=n) for k in range(flat.shape[1])], axis=1)
    return out.reshape((n,) + vals.shape[1:])


def reference_pairs(x0: np.ndarray, h: float):
    """Directed pairs (a, b), a != b, with |r0_a - r0_b| < 2h (fixed for the whole run)."""
    t = cKDTree(x0)
    pp = t.query_pairs(2.0 * h * (1.0 + 1e-9), output_type="ndarray")
    if pp.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    I = np.concatenate([pp[:, 0], pp[:, 1]]).astype(np.int64)
    J = np.concatenate([pp[:, 1], pp[:, 0]]).astype(np.int64)
    d = x0[I] - x0[J]
    keep = np.sum(d * d, axis=1) < (2.0 * h) ** 2
    return I[keep], J[keep]


def reference_gradients(x0, I, J, h, dim):
    """grad0_a W_ab = dW/dr(|r0_ab|) r0_ab / |r0_ab| (R2)."""
    r = x0[I] - x0[J]
    dist = np.sqrt(np.sum(r * r, axis=1))
    return (o.kernel_dW(dist, h, dim) / dist)[:, None] * r


def correction_matrix(x0, V, I, J, gW):
    """Eq. sph-correctmatrix: B0_a = (sum_b V_b (r0_b - r0_a) (x) grad0_a W_ab)^-1."""
    N, d = x0.shape
    outer = (V[J][:, None] * (x0[J] - x0[I]))[:, :, None] * gW[:, None, :]
    return np.linalg.inv(_scatter(I, outer, N))


def make_solid(x0, V, n, fixed, mat: Material, h: float, gravity) -> Solid:
    x0 = np.asarray(x0, dtype=np.float64)
    d = x0.shape[1]
    I, J = reference_pairs(x0, h)
    gW = reference_gradients(x0, I, J, h, d)
    B0 = correction_matrix(x0, np.asarray(V, dtype=np.float64), I, J, gW)
    N = x0.shape[0]
    eye = np.broadcast_to(np.eye(d), (N, d, d)).copy()
    z = np.zeros((N, d))
    return Solid(x0=x0, x=x0.copy(), v=z.copy(), F=eye, dFdt=np.zeros((N, d, d)),
                 V=np.asarray(V, dtype=np.float64).copy(), n=np.asarray(n, dtype=np.float64).copy(),
                 fixed=np.asarray(fixed, dtype=bool).copy(), B0=B0, I=I, J=J, gW=gW, mat=mat, h=float(h),
                 gravity=np.asarray(gravity, dtype=np.float64)[:d].copy(), acc=z.copy(), vbar=z.copy(),
                 abar=z.copy(), f_fluid=z.copy())


def deformation_gradient_from_displacement(sol: Solid, u: np.ndarray) -> np.ndarray:
    """F = (sum_b V_b (u_b - u_a) (x) grad0_a W_ab) B0_a + I (the paper's definition of F)."""
    N, d = sol.x0.shape
    outer = (sol.V[sol.J][:, None] * (u[sol.J] - u[sol.I]))[:, :, None] * sol.gW[:, None, :]
    return _scatter(sol.I, outer, N) @ sol.B0 + np.eye(d)


def deformation_rate(sol: Solid) -> np.ndarray:
    """R20: dF/dt = (sum_b V_b (v_b - v_a) (x) grad0_a W_ab) B0_a."""
    N, d = sol.x0.shape
    outer = (sol.V[sol.J][:, None] * (sol.v[sol.J] - sol.v[sol.I]))[:, :, None] * sol.gW[:, None, :]
    return _scatter(sol.I, outer, N) @ sol.B0


def first_piola(F: np.ndarray, mat: Material) -> np.ndarray:
    """P = F S. Linear: S = lambda tr(E) I + 2 mu E, E = (F^T F - I)/2. Neo-Hookean
    (W = mu tr E - mu ln J + lambda/2 (ln J)^2): S = mu (I - C^-1) + lambda ln J C^-1."""
    d = F.shape[-1]
    eye = np.eye(d)
    C = np.swapaxes(F, -1, -2) @ F
    if mat.model == LINEAR:
        E = 0.5 * (C - eye)
        trE = np.trace(E, axis1=-2, axis2=-1)
        S = mat.lam * trE[:, None, None] * eye + 2.0 * mat.mu * E
    elif mat.model == NEO_HOOKEAN:
        Cinv = np.linalg.inv(C)
        lnJ = np.log(np.linalg.det(F))
        S = mat.mu * (eye - Cinv) + mat.lam * lnJ[:, None, None] * Cinv
    else:
        raise ValueError("unknown material model")
    return F @ S


def elastic_acceleration(sol: Solid) -> np.ndarray:
    """Eq. sph-mechanical-mom without g: (2/m_a) sum_b V_a V_b P~_ab grad0_a W_ab,
    P~_ab = (P_a B0_a + P_b B0_b)/2."""
    N, d = sol.x0.shape
    PB = first_piola(sol.F, sol.mat) @ sol.B0
    Pt = 0.5 * (PB[sol.I] + PB[sol.J])
    term = (sol.V[sol.I] * sol.V[sol.J])[:, None] * np.einsum("kij,kj->ki", Pt, sol.gW)
    return 2.0 * _scatter(sol.I, term, N) / sol.m[:, None]


def solid_dt(sol: Solid) -> float:
    """Eq. dts-advection: 0.6 min(h / (c + |v|max), sqrt(h / |dv/dt|max))."""
    vmax = float(np.sqrt(np.max(np.sum(sol.v * sol.v, axis=1)))) if sol.v.size else 0.0
    amax = float(np.sqrt(np.max(np.sum(sol.acc * sol.acc, axis=1)))) if sol.acc.size else 0.0
    dt = sol.h / (sol.mat.c + vmax)
    if amax > 0.0:
        dt = min(dt, math.sqrt(sol.h / amax))
    return 0.6 * dt


def solid_step(sol: Solid, dt: float) -> np.ndarray:
    """One solid step (Eqs. verlet-first-half-solid, verlet-first-mediate-solid,
    verlet-first-final-solid) with the held fluid force; returns dv/dt."""
    free = ~sol.fixed
    sol.F = sol.F + 0.5 * dt * sol.dFdt
    sol.x[free] = sol.x[free] + 0.5 * dt * sol.v[free]
    acc = elastic_acceleration(sol) + sol.gravity[None, :] + sol.f_fluid / sol.m[:, None]
    acc[sol.fixed] = 0.0
    sol.v = sol.v + dt * acc
    sol.v[sol.fixed] = 0.0
    sol.x[free] = sol.x[free] + 0.5 * dt * sol.v[free]
    sol.dFdt = deformation_rate(sol)
    sol.F = sol.F + 0.5 * dt * sol.dFdt
    sol.acc = acc
    return acc


# --------------------------------------------------------------------------------------
# Fluid-structure coupling (fluid kernel h_F)
# --------------------------------------------------------------------------------------
def coupling_pairs(xf: np.ndarray, xs: np.ndarray, prm: o.Params):
    """(fluid i, solid a) pairs with |r_i - r_a| < 2 h_F."""
    if xf.shape[0] == 0 or xs.shape[0] == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z
    tf, ts = cKDTree(xf), cKDTree(xs)
    sm = tf.sparse_distance_matrix(ts, 2.0 * prm.h * (1.0 + 1e-9), output_type="ndarray")
    I, A = sm["i"].astype(np.int64), sm["j"].astype(np.int64)
    d = xf[I] - xs[A]
    keep = np.sum(d * d, axis=1) < (2.0 * prm.h) ** 2
    return I[keep], A[keep]


def imaginary_pressure(p_i, rho_i, r_ia, n_a, abar_a, g):
    """R22: p^d = p_i + rho_i max(0, -(g - a~).n) ((r_i - r_a).n)."""
    proj = np.maximum(0.0, -np.sum((g[None, :] - abar_a) * n_a, axis=1))
    return p_i + rho_i * proj * np.sum(r_ia * n_a, axis=1)


def coupling_forces(x, rho, v, m, sol: Solid, prm: o.Params):
    """Fluid pressure and viscous forces between the fluid (positions x, densities rho,
    velocities v, masses m) and the solid at its current positions (Eqs. fs-force-mr-sp,
    fs-force-mr-sv with R21-R23). Returns (the fluid's dv/dt contribution (N, d), the force
    on the solid (Ns, d)); the two are equal and opposite pair by pair."""
    N, d = x.shape
    Ns = sol.x.shape[0]
    I, A = coupling_pairs(x, sol.x, prm)
    acc = np.zeros((N, d))
    force = np.zeros((Ns, d))
    if I.size == 0:
        return acc, force
    r = x[I] - sol.x[A]
    dist = np.sqrt(np.sum(r * r, axis=1))
    dW = o.kernel_dW(dist, prm.h, d)
    grad = np.where((dist > 0.0)[:, None], (dW / np.where(dist > 0, dist, 1.0))[:, None] * r, 0.0)
    p = o.eos_pressure(rho, prm)
    pd = imaginary_pressure(p[I], rho[I], r, sol.n[A], sol.abar[A], prm.gravity)
    rhod = prm.rho0 + pd / prm.c0 ** 2
    pbar = (p[I] * rhod + pd * rho[I]) / (rho[I] + rhod)
    V_i = m[I] / rho[I]
    f = (-2.0 * V_i * sol.V[A] * pbar)[:, None] * grad                  # Eq. fs-force-mr-sp
    if prm.nu > 0.0:
        eta = prm.rho0 * prm.nu
        vd = 2.0 * sol.vbar[A] - v[I]                                    # R23
        f += (2.0 * eta * V_i * sol.V[A] / (dist + 0.01 * prm.h) * dW)[:, None] * (v[I] - vd)
    acc = _scatter(I, f / m[I][:, None], N)
    force = _scatter(A, -f, Ns)
    return acc, force


def coupling_continuity(x, rho, v, sol: Solid, prm: o.Params) -> np.ndarray:
    """R28: d rho/dt of fluid particles from their solid neighbours, each a moving wall."""
    N, d = x.shape
    I, A = coupling_pairs(x, sol.x, prm)
    if I.size == 0:
        return np.zeros(N)
    r = x[I] - sol.x[A]
    dist = np.sqrt(np.sum(r * r, axis=1))
    dW = o.kernel_dW(dist, prm.h, d)
    n = sol.n[A]
    UL = -np.sum(n * v[I], axis=1)
    uw = -np.sum(n * sol.vbar[A], axis=1)
    UR = -UL + 2.0 * uw
    p = o.eos_pressure(rho, prm)
    PL = p[I]
    PR = imaginary_pressure(PL, rho[I], r, n, sol.abar[A], prm.gravity)
    rhoR = prm.rho0 + PR / prm.c0 ** 2
    Us, _ = o.riemann(rho[I], rhoR, UL, UR, PL, PR, prm.c0)
    return _scatter(I, 2.0 * rho[I] * sol.V[A] * (Us - UL) * dW, N)


def solid_substeps(sol: Solid, dt_f: float) -> int:
    """R24, R25: kappa = [dt_F / dt_S] + 1 solid steps of dt_F / kappa with the held fluid
    force; v~ and a~ become their averages. Returns kappa."""
    kappa = int(math.floor(dt_f / solid_dt(sol))) + 1
    h = dt_f / kappa
    vsum = np.zeros_like(sol.v)
    asum = np.zeros_like(sol.v)
    for _ in range(kappa):
        asum += solid_step(sol, h)
        vsum += sol.v
    sol.vbar = vsum / kappa
    sol.abar = asum / kappa
    return kappa


def acoustic_substep(st: o.State, w: o.Walls, nb, acc_prior, dt: float, prm: o.Params, sol: Solid):
    """One fluid acoustic step of the coupled system (R26). The solid is updated in place.
    Returns (fluid state, fluid dv/dt, kappa)."""
    half, dvdt = o.pressure_relaxation(st, w, nb, acc_prior, dt, prm)
    a_fsi, f_solid = coupling_forces(half.x, half.rho, st.v, st.m, sol, prm)
    half.v = half.v + dt * a_fsi
    dvdt = dvdt + a_fsi
    out = o.density_relaxation(half, w, nb, dt, prm)
    drho = coupling_continuity(out.x, half.rho, out.v, sol, prm)
    out.rho = out.rho + 0.5 * dt * drho
    out.drho = out.drho + drho
    out.t = st.t + dt
    sol.f_fluid = f_solid
    kappa = solid_substeps(sol, dt)
    return out, dvdt, kappa


def advection_step(st: o.State, w: o.Walls, prm: o.Params, sol: Solid):
    """One dual-criteria step of the coupled system: the fluid's neighbour set, Dt_ad and
    density re-initialisation (R30: solid particles take no part in it, so fluid next to the
    solid keeps its continuity density through the free-surface max), then acoustic steps
    with the solid until Dt_ad is covered. Returns (state, substeps, solid steps)."""
    st = st.copy()
    nb = o.neighbour_sets(st.x, w.x, prm)
    Dt = o.dt_advection(st.v, prm)
    st.rho = o.density_summation(st, w, nb, prm)
    acc_prior = o.viscous_acceleration(st, nb, prm)
    tau, sub, solid_steps = 0.0, 0, 0
    while tau < Dt * (1.0 - o.LOOP_SLACK):
        dt = min(o.dt_acoustic(st.v, prm), Dt - tau)
        st, _, kappa = acoustic_substep(st, w, nb, acc_prior, dt, prm, sol)
        tau += dt
        sub += 1
        solid_steps += kappa
    return st, sub, solid_steps


def solid_from_problem(p) -> Solid:
    """The solid of a workload carrying solid_* attributes."""
    mat = Material(rho0=p.solid_rho0, youngs=p.solid_youngs, poisson=p.solid_poisson, model=p.solid_model)
    return make_solid(p.solid_pos, p.solid_vol, p.solid_normal, p.solid_fixed, mat, p.solid_h, p.gravity)
