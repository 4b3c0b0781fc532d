"""Plain FP64 CPU oracle of the Riemann-solver WCSPH hot path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use this
module. It shares no code with the CUDA library.

The method (paper Sec. 1.1, 2.1-2.4, 6 "position-based Verlet"), in the paper's order:

  * Wendland C2 kernel with support 2h (kernel_wenland_c2, Sec. 6.2 table; Wendland 1995).
  * Neighbour set of an advection step: all j != i with |r_i - r_j| < 2h (cell-linked
    list, Sec. 6.2); frozen for that step's acoustic substeps (Sec. 2.4: the advection
    criterion fixes how often the particle configuration is updated).
  * Density re-initialisation at the start of each advection step (Eq. eqrhosum,
    Eq. eqrhosumnosurface), viscous acceleration (Eq. eqviscous).
  * Dual-criteria time steps (Eq. dt-advection, Eq. dt-relax).
  * Per acoustic substep: pressure relaxation (Eq. verlet-first-half, Eq. eqeos,
    Eq. riemannsph momentum with the wall problem of Eqs. eqriepartial, eqrienoslip,
    eqriepright, then Eq. verlet-first-mediate) and density relaxation
    (Eq. verlet-first-final with Eq. riemannsph continuity).

Readings where the paper is silent or inconsistent (the same readings the CUDA path takes):
  R1  Wendland C2 is W = alpha_d (1 - q/2)^4 (1 + 2q), q = r/h < 2, alpha_2 = 7/(4 pi h^2),
      alpha_3 = 21/(16 pi h^3) (the formula is only cited, Sec. 6.2).
  R2  Sign convention: r_ij = r_i - r_j, e_ij = -r_ij/|r_ij| points from i to j (Sec. 2.2),
      and grad_i W_ij = dW/dr * r_ij/|r_ij| (the true gradient; Sec. 1.1 writes it with e_ij,
      which would flip the sign of the momentum equation).
  R3  Riemann solver: the cited low-dissipation solver, not printed in the paper:
      U* = (U_L+U_R)/2 + (P_L-P_R)/(2 rho_bar c0), P* = (P_L+P_R)/2 + rho_bar c0 beta (U_L-U_R)/2,
      rho_bar = (rho_L+rho_R)/2, beta = min(LIMITER * max(U_L-U_R, 0)/c0, 1), LIMITER = 3.
  R4  Wall pair: U_L = -n_w.v_i, U_R = -U_L (static wall), P_L = p_i, P_R = p_i + rho_i g.(r_w - r_i),
      rho_R from the EoS; the continuity term uses (U* - U_L) in place of (U* - v_i.e_ij);
      wall volume V_w replaces m_j/rho_j.
  R5  sum W^0 is the full-lattice sum including self at spacing dp (a constant).
      Walls count in sum W with weight 1. Self term W(0) is included.
  R6  Pair geometry is recomputed from current positions in every half step; pairs that
      drift beyond 2h contribute nothing; pairs that come within 2h are ignored until the
      next advection step. Pairs at zero distance contribute nothing.
  R7  Delta t_ad uses max(|v|max, U_ref) with U_ref = c0/10 (c = 10 U_max, Sec. 2.1) and
      drops the h^2/nu term when nu = 0; the acoustic substep is clamped to the remainder
      of the advection step; the loop runs while tau < Dt_ad (1 - 1e-12).
  R8  Viscous acceleration is fluid-fluid only, with eta = rho0 nu, evaluated once per
      advection step after density re-initialisation and held over its substeps.
  R9  In the second half step the position update uses v^{n+1}.
  R10 Particles are stored in (search cell, id) order, search cells being the 2h position
      cells halved on every axis and flattened x fastest (Sec. 6.2 fixes no order inside the
      cell-linked list); neighbour sets are those of the 2h definition.
  R11 Optional frozen pair geometry: r_i - r_j and (dW/dr)/r of every pair taken at the
      configuration update and used by every half step of the advection step.
  R12 Transport velocity (Eq. transport, flows without free surface), off when p0 = 0: the
      background-pressure acceleration a_i = -2 sum_j m_j p0/(rho_i rho_j) grad_i W_ij over
      fluid pairs, with the mid-point geometry and densities of the pressure relaxation, acts
      on the transport velocity only; the transport velocity starts each substep equal to v,
      so over the substep it moves the particle by dt^2/2 a_i in addition to v, applied to
      the mid-point position. p0 is not given in the paper: 2 rho0 c0^2 for the Taylor-Green
      vortex (the largest value that stayed stable in a sweep at 40^2).

  R18 Particle gradients (Eqs. gradsph-strong, gradsph-weak): the paper's grad_i W_ij there
      is e_ij dW/dr with e_ij from i to j, minus the true gradient of R2; with the true
      gradient the strong form is sum_j V_j (f_j - f_i) grad_i W_ij and the weak form
      sum_j V_j (f_i + f_j) grad_i W_ij. Wall neighbours carry the wall problem's p and rho (R4).

Parity pins: every function here is pinned by the tests in tests/test_oracle_pins.py and
tests/test_gradient_oracle.py (closed forms, invariants, brute force). None is unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

LIMITER = 3.0               # R3: dissipation-limiter constant
LOOP_SLACK = 1e-12          # R7: relative slack of the substep loop condition
QUANT_BITS = 22             # fixed-point bits per cell (position representation contract)


# --------------------------------------------------------------------------------------
# Wendland C2 kernel (R1)
# --------------------------------------------------------------------------------------
def wendland_alpha(h: float, dim: int) -> float:
    if dim == 2:
        return 7.0 / (4.0 * math.pi * h * h)
    if dim == 3:
        return 21.0 / (16.0 * math.pi * h ** 3)
    raise ValueError("dim must be 2 or 3")


def kernel_W(r, h, dim):
    """W(r, h) with compact support 2h."""
    q = np.asarray(r, dtype=np.float64) / h
    t = np.clip(1.0 - 0.5 * q, 0.0, None)
    return wendland_alpha(h, dim) * t ** 4 * (1.0 + 2.0 * q)


def kernel_dW(r, h, dim):
    """dW/dr (negative inside the support, zero beyond 2h)."""
    q = np.asarray(r, dtype=np.float64) / h
    t = np.clip(1.0 - 0.5 * q, 0.0, None)
    return wendland_alpha(h, dim) / h * (-5.0 * q) * t ** 3


def lattice_sigma0(dp: float, h: float, dim: int) -> float:
    """R5: sum over an infinite square/cubic lattice of W(|k| dp), self included."""
    kmax = int(math.ceil(2.0 * h / dp)) + 1
    ax = np.arange(-kmax, kmax + 1, dtype=np.float64)
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    r = dp * np.sqrt(sum(g * g for g in grids))
    return float(np.sum(kernel_W(r, h, dim)))


# --------------------------------------------------------------------------------------
# Parameters and state
# --------------------------------------------------------------------------------------
@dataclass
class Params:
    dim: int
    h: float
    dp: float
    rho0: float
    c0: float
    cfl_ad: float
    cfl_ac: float
    u_ref: float
    nu: float
    gravity: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    periodic: np.ndarray
    free_surface: bool
    sigma0: float = 0.0
    p_transport: float = 0.0   # R12: background pressure p0 of Eq. transport (0 = off)

    @staticmethod
    def from_problem(p) -> "Params":
        """Read the parameters from any object carrying the problem's attributes."""
        d = int(p.dim)
        prm = Params(dim=d, h=float(p.h), dp=float(p.dp), rho0=float(p.rho0), c0=float(p.c0),
                     cfl_ad=float(p.cfl_ad), cfl_ac=float(p.cfl_ac), u_ref=float(p.u_ref),
                     nu=float(p.nu), gravity=np.asarray(p.gravity, dtype=np.float64)[:d].copy(),
                     lo=np.asarray(p.lo, dtype=np.float64)[:d].copy(),
                     hi=np.asarray(p.hi, dtype=np.float64)[:d].copy(),
                     periodic=np.asarray(p.periodic)[:d].astype(bool),
                     free_surface=bool(p.free_surface),
                     p_transport=float(getattr(p, "p_transport", 0.0)))
        prm.sigma0 = lattice_sigma0(prm.dp, prm.h, d)
        return prm

    @property
    def period(self) -> np.ndarray:
        """Period length per axis (0 on non-periodic axes)."""
        return np.where(self.periodic, self.hi - self.lo, 0.0)


@dataclass
class State:
    x: np.ndarray          # (N, d) positions
    v: np.ndarray          # (N, d) velocities
    rho: np.ndarray        # (N,) densities
    drho: np.ndarray       # (N,) d rho/dt carried between substeps
    m: np.ndarray          # (N,) masses (never written)
    t: float = 0.0

    def copy(self) -> "State":
        return State(self.x.copy(), self.v.copy(), self.rho.copy(), self.drho.copy(),
                     self.m.copy(), self.t)


@dataclass
class Walls:
    x: np.ndarray          # (Nw, d)
    n: np.ndarray          # (Nw, d) unit normals into the fluid
    V: np.ndarray          # (Nw,) volumes


def state_from_problem(p) -> tuple[State, Walls]:
    d = int(p.dim)
    st = State(np.array(p.pos, dtype=np.float64).reshape(-1, d),
               np.array(p.vel, dtype=np.float64).reshape(-1, d),
               np.array(p.rho, dtype=np.float64).copy(),
               np.zeros(len(p.rho)), np.array(p.mass, dtype=np.float64).copy(), 0.0)
    w = Walls(np.array(p.wall_pos, dtype=np.float64).reshape(-1, d),
              np.array(p.wall_normal, dtype=np.float64).reshape(-1, d),
              np.array(p.wall_vol, dtype=np.float64).copy())
    return st, w


# --------------------------------------------------------------------------------------
# Neighbour sets (cell-linked list replaced by the plain definition)
# --------------------------------------------------------------------------------------
def min_image(d: np.ndarray, period: np.ndarray) -> np.ndarray:
    """Minimum-image difference vectors on periodic axes (period 0 = not periodic)."""
    out = d.copy()
    for a in range(d.shape[1]):
        L = period[a]
        if L > 0:
            out[:, a] -= L * np.round(out[:, a] / L)
    return out


def _tree(x: np.ndarray, prm: Params):
    """KD-tree over positions; periodic axes wrap, other axes get a box too large to wrap."""
    per = prm.period
    span = prm.hi - prm.lo
    box = np.where(per > 0, per, 4.0 * span + 1.0)
    xs = x - prm.lo
    xs = np.where(per > 0, np.mod(xs, np.where(per > 0, per, 1.0)), xs + 1.5 * span)
    return cKDTree(xs, boxsize=box)


def brute_force_pairs(xa: np.ndarray, xb: np.ndarray, radius: float, period: np.ndarray,
                      same: bool):
    """All (i, j) with |xa_i - xb_j| < radius by testing every pair (tiny inputs only)."""
    I, J = [], []
    for i in range(xa.shape[0]):
        d = min_image(xa[i][None, :] - xb, period)
        r2 = np.sum(d * d, axis=1)
        js = np.nonzero(r2 < radius * radius)[0]
        if same:
            js = js[js != i]
        I.extend([i] * len(js))
        J.extend(js.tolist())
    return np.asarray(I, dtype=np.int64), np.asarray(J, dtype=np.int64)


def candidate_pairs(x: np.ndarray, xw: np.ndarray, radius: float, prm: Params):
    """Directed fluid-fluid pairs (both orders) and fluid-wall pairs within `radius` (<=)."""
    tf = _tree(x, prm)
    pp = tf.query_pairs(radius, output_type="ndarray")
    if pp.size == 0:
        I = J = np.zeros(0, dtype=np.int64)
    else:
        I = np.concatenate([pp[:, 0], pp[:, 1]]).astype(np.int64)
        J = np.concatenate([pp[:, 1], pp[:, 0]]).astype(np.int64)
    if xw.shape[0] and x.shape[0]:
        tw = _tree(xw, prm)
        sm = tf.sparse_distance_matrix(tw, radius, output_type="ndarray")
        IW = sm["i"].astype(np.int64)
        KW = sm["j"].astype(np.int64)
    else:
        IW = KW = np.zeros(0, dtype=np.int64)
    return I, J, IW, KW


def neighbour_sets(x: np.ndarray, xw: np.ndarray, prm: Params):
    """Frozen neighbour set of an advection step: |r_i - r_j| < 2h, j != i (FP64 test)."""
    R = 2.0 * prm.h
    I, J, IW, KW = candidate_pairs(x, xw, R * (1.0 + 1e-9), prm)
    d = min_image(x[I] - x[J], prm.period)
    keep = np.sum(d * d, axis=1) < R * R
    I, J = I[keep], J[keep]
    if IW.size:
        dw = x[IW] - xw[KW]
        keepw = np.sum(dw * dw, axis=1) < R * R
        IW, KW = IW[keepw], KW[keepw]
    return I, J, IW, KW


# --- Fixed-point position contract (shared specification, independent implementation) ---
def quantisation(prm: Params):
    """Cell size, cells per axis, bits per cell and quantum of the position contract.

    Cell size is 2h, or period/floor(period/2h) when an axis is periodic (all periodic
    axes share one period). Positions are integers q = rint((x - lo)/dq) with
    dq = cell/2^bits, bits = min(22, 31 - bitlength(max cells per axis)).
    """
    d = prm.dim
    per = prm.period
    if np.any(per > 0):
        L = float(per[per > 0][0])
        cell = L / math.floor(L / (2.0 * prm.h))
    else:
        cell = 2.0 * prm.h
    ncell = []
    for a in range(d):
        if per[a] > 0:
            ncell.append(int(math.floor(per[a] / (2.0 * prm.h))))
        else:
            ncell.append(max(1, int(math.ceil((prm.hi[a] - prm.lo[a]) / cell))))
    bits = min(QUANT_BITS, 31 - max(ncell).bit_length())
    dq = cell / float(1 << bits)
    x = 2.0 * prm.h / dq
    R2 = int(math.ceil(x * x))
    return cell, ncell, bits, dq, R2


def quantise(x: np.ndarray, prm: Params) -> np.ndarray:
    cell, ncell, bits, dq, _ = quantisation(prm)
    q = np.rint((x - prm.lo[None, :]) / dq).astype(np.int64)
    for a in range(prm.dim):
        if prm.periodic[a]:
            q[:, a] = np.mod(q[:, a], ncell[a] << bits)
    return q


def dequantise(q: np.ndarray, prm: Params) -> np.ndarray:
    _, _, _, dq, _ = quantisation(prm)
    return prm.lo[None, :] + q.astype(np.float64) * dq


def neighbour_sets_quantised(x: np.ndarray, xw: np.ndarray, prm: Params):
    """Neighbour sets decided on the fixed-point positions: sum dq_a^2 < R2 (integers)."""
    cell, ncell, bits, dq, R2 = quantisation(prm)
    I, J, IW, KW = candidate_pairs(x, xw, 2.0 * prm.h + 4.0 * dq, prm)
    qf = quantise(x, prm)
    per_q = np.array([(ncell[a] << bits) if prm.periodic[a] else 0 for a in range(prm.dim)],
                     dtype=np.int64)

    def d2(qa, qb):
        dd = qa - qb
        for a in range(prm.dim):
            if per_q[a]:
                P = per_q[a]
                dd[:, a] = np.mod(dd[:, a] + P // 2, P) - P // 2
        return np.sum(dd * dd, axis=1)

    keep = d2(qf[I], qf[J]) < R2
    I, J = I[keep], J[keep]
    if IW.size:
        qw = quantise(xw, prm)
        keepw = d2(qf[IW], qw[KW]) < R2
        IW, KW = IW[keepw], KW[keepw]
    return I, J, IW, KW


def cell_permutation(x: np.ndarray, ids: np.ndarray, prm: Params) -> np.ndarray:
    """Particle ids in (search cell, id) order. Search cells halve the position cell on
    every axis (cell index q >> (bits - 1), about h wide) and are flattened with x fastest;
    the order is the one the cell-linked list of Sec. 6.2 is stored in (reading R10)."""
    cell, ncell, bits, dq, _ = quantisation(prm)
    c = quantise(x, prm) >> (bits - 1)
    flat = np.zeros(x.shape[0], dtype=np.int64)
    stride = 1
    for a in range(prm.dim):
        flat += c[:, a] * stride
        stride *= 2 * ncell[a]
    order = np.lexsort((ids, flat))
    return ids[order]


# --------------------------------------------------------------------------------------
# Riemann solver (R3) and equation of state (Eq. eqeos)
# --------------------------------------------------------------------------------------
def eos_pressure(rho, prm: Params):
    return prm.c0 ** 2 * (rho - prm.rho0)


def riemann(rhoL, rhoR, UL, UR, PL, PR, c0):
    """Interface velocity U* and pressure P* of the inter-particle Riemann problem."""
    rho_bar = 0.5 * (rhoL + rhoR)
    beta = np.minimum(LIMITER * np.maximum(UL - UR, 0.0) / c0, 1.0)
    Ustar = 0.5 * (UL + UR) + (PL - PR) / (2.0 * rho_bar * c0)
    Pstar = 0.5 * (PL + PR) + 0.5 * rho_bar * c0 * beta * (UL - UR)
    return Ustar, Pstar


def _geometry(xa, xb, prm: Params):
    """r_ij = r_i - r_j (minimum image), |r_ij|, and e_ij = -r_ij/|r_ij| (zero at r = 0)."""
    rij = min_image(xa - xb, prm.period)
    r = np.sqrt(np.sum(rij * rij, axis=1))
    safe = np.where(r > 0.0, r, 1.0)
    e = np.where((r > 0.0)[:, None], -rij / safe[:, None], 0.0)
    return rij, r, e


def _from_rij(rij):
    """|r_ij| and e_ij = -r_ij/|r_ij| of given pair vectors (as _geometry returns them)."""
    r = np.sqrt(np.sum(rij * rij, axis=1))
    safe = np.where(r > 0.0, r, 1.0)
    e = np.where((r > 0.0)[:, None], -rij / safe[:, None], 0.0)
    return rij, r, e


def frozen_geometry(st: State, w: Walls, nb, prm: Params):
    """Pair vectors r_i - r_j (minimum image) of the fluid and the wall pairs at the
    configuration update, kept for the whole advection step (reading R11: Sec. 2.4 and
    Sec. 6.2 store the pair geometry in the neighbour relation when it is built)."""
    I, J, IW, KW = nb
    rij = _geometry(st.x[I], st.x[J], prm)[0]
    rfw = _geometry(st.x[IW], w.x[KW], prm)[0]
    return rij, rfw


def _scatter_add(idx, vals, n):
    if vals.ndim == 1:
        return np.bincount(idx, weights=vals, minlength=n)
    return np.stack([np.bincount(idx, weights=vals[:, a], minlength=n)
                     for a in range(vals.shape[1])], axis=1)


# --------------------------------------------------------------------------------------
# Advection-step operations
# --------------------------------------------------------------------------------------
def density_summation(st: State, w: Walls, nb, prm: Params) -> np.ndarray:
    """Eq. eqrhosum (free surface) / Eq. eqrhosumnosurface: rho0 * sum W / sum W^0."""
    I, J, IW, KW = nb
    N = st.x.shape[0]
    _, r, _ = _geometry(st.x[I], st.x[J], prm)
    sumW = kernel_W(0.0, prm.h, prm.dim) + _scatter_add(I, kernel_W(r, prm.h, prm.dim), N)
    if IW.size:
        _, rw, _ = _geometry(st.x[IW], w.x[KW], prm)
        sumW = sumW + _scatter_add(IW, kernel_W(rw, prm.h, prm.dim), N)
    rho_sum = prm.rho0 * sumW / prm.sigma0
    if prm.free_surface:
        return np.maximum(st.rho, rho_sum)
    return rho_sum


def viscous_acceleration(st: State, nb, prm: Params) -> np.ndarray:
    """Eq. eqviscous with eta = rho0 nu over fluid neighbours (R8)."""
    I, J, _, _ = nb
    N = st.x.shape[0]
    d = prm.dim
    if prm.nu == 0.0 or I.size == 0:
        return np.zeros((N, d))
    eta = prm.rho0 * prm.nu
    _, r, _ = _geometry(st.x[I], st.x[J], prm)
    dW = kernel_dW(r, prm.h, prm.dim)
    safe = np.where(r > 0.0, r, 1.0)
    coef = np.where(r > 0.0, 2.0 * st.m[J] * eta / (st.rho[I] * st.rho[J]) * dW / safe, 0.0)
    return _scatter_add(I, coef[:, None] * (st.v[I] - st.v[J]), N)


def dt_advection(v: np.ndarray, prm: Params) -> float:
    """Eq. dt-advection with the U_ref floor of R7."""
    vmax = float(np.sqrt(np.max(np.sum(v * v, axis=1)))) if v.size else 0.0
    dt = prm.h / max(vmax, prm.u_ref)
    if prm.nu > 0.0:
        dt = min(dt, prm.h * prm.h / prm.nu)
    return prm.cfl_ad * dt


def dt_acoustic(v: np.ndarray, prm: Params) -> float:
    """Eq. dt-relax."""
    vmax = float(np.sqrt(np.max(np.sum(v * v, axis=1)))) if v.size else 0.0
    return prm.cfl_ac * prm.h / (prm.c0 + vmax)


def pressure_relaxation(st: State, w: Walls, nb, acc_prior, dt: float, prm: Params,
                        geometry=None):
    """First half of the position-based Verlet substep.

    Eq. verlet-first-half: rho and r to the mid point; Eq. eqeos: pressure;
    Eq. riemannsph (momentum) for fluid pairs and the one-sided wall problem
    (Eqs. eqriepartial, eqrienoslip, eqriepright) for wall pairs;
    Eq. verlet-first-mediate: v to the new step. Returns (state, dv/dt).
    With `geometry` (from frozen_geometry) the pair vectors are those of the
    configuration update instead of the mid-point positions (reading R11).
    With a background pressure p0 > 0 (Eq. transport, reading R12) the mid-point
    position also takes the transport shift dt^2/2 a_i.
    """
    I, J, IW, KW = nb
    N = st.x.shape[0]
    c0, g = prm.c0, prm.gravity
    rho = st.rho + 0.5 * dt * st.drho
    x = st.x + 0.5 * dt * st.v
    p = eos_pressure(rho, prm)
    acc = np.zeros((N, prm.dim))
    shift = 0.0
    if I.size:
        rij, r, e = _geometry(x[I], x[J], prm) if geometry is None else _from_rij(geometry[0])
        dW = kernel_dW(r, prm.h, prm.dim)
        UL = np.sum(st.v[I] * e, axis=1)
        UR = np.sum(st.v[J] * e, axis=1)
        _, Ps = riemann(rho[I], rho[J], UL, UR, p[I], p[J], c0)
        grad = (-e) * dW[:, None]                    # grad_i W_ij = dW/dr r_ij/|r_ij|  (R2)
        Vj = st.m[J] / rho[J]
        acc += _scatter_add(I, (-2.0 * Vj * Ps / rho[I])[:, None] * grad, N)
        if prm.p_transport > 0.0:
            # Eq. transport: -2 sum_j m_j p0 / (rho_i rho_j) grad_i W_ij (R12)
            a_tv = _scatter_add(I, (-2.0 * prm.p_transport * Vj / rho[I])[:, None] * grad, N)
            shift = 0.5 * dt * dt * a_tv
    if IW.size:
        if geometry is None:
            rfw, r, e = _geometry(x[IW], w.x[KW], prm)
        else:
            rfw, r, e = _from_rij(geometry[1])
        dW = kernel_dW(r, prm.h, prm.dim)
        UL = -np.sum(w.n[KW] * st.v[IW], axis=1)
        UR = -UL
        PL = p[IW]
        PR = PL + rho[IW] * ((-rfw) @ g)              # r_w - r_f = -(r_f - r_w)
        rhoR = prm.rho0 + PR / c0 ** 2
        _, Ps = riemann(rho[IW], rhoR, UL, UR, PL, PR, c0)
        grad = (-e) * dW[:, None]
        acc += _scatter_add(IW, (-2.0 * w.V[KW] * Ps / rho[IW])[:, None] * grad, N)
    dvdt = acc_prior + g[None, :] + acc
    v = st.v + dt * dvdt
    out = State(x + shift, v, rho, st.drho.copy(), st.m, st.t)
    return out, dvdt


def density_relaxation(st: State, w: Walls, nb, dt: float, prm: Params, geometry=None):
    """Second half of the substep: Eq. verlet-first-final with the continuity equation
    of Eq. riemannsph (fluid pairs) and its one-sided wall form (R4). Returns state.
    With `geometry` the pair vectors are the frozen ones (reading R11)."""
    I, J, IW, KW = nb
    N = st.x.shape[0]
    c0, g = prm.c0, prm.gravity
    x = st.x + 0.5 * dt * st.v                      # R9: v here is v^{n+1}
    rho = st.rho
    p = eos_pressure(rho, prm)
    drho = np.zeros(N)
    if I.size:
        _, r, e = _geometry(x[I], x[J], prm) if geometry is None else _from_rij(geometry[0])
        dW = kernel_dW(r, prm.h, prm.dim)
        UL = np.sum(st.v[I] * e, axis=1)
        UR = np.sum(st.v[J] * e, axis=1)
        Us, _ = riemann(rho[I], rho[J], UL, UR, p[I], p[J], c0)
        Vj = st.m[J] / rho[J]
        drho += _scatter_add(I, 2.0 * rho[I] * Vj * (Us - UL) * dW, N)
    if IW.size:
        if geometry is None:
            rfw, r, e = _geometry(x[IW], w.x[KW], prm)
        else:
            rfw, r, e = _from_rij(geometry[1])
        dW = kernel_dW(r, prm.h, prm.dim)
        UL = -np.sum(w.n[KW] * st.v[IW], axis=1)
        UR = -UL
        PL = p[IW]
        PR = PL + rho[IW] * ((-rfw) @ g)
        rhoR = prm.rho0 + PR / c0 ** 2
        Us, _ = riemann(rho[IW], rhoR, UL, UR, PL, PR, c0)
        drho += _scatter_add(IW, 2.0 * rho[IW] * w.V[KW] * (Us - UL) * dW, N)
    rho_new = rho + 0.5 * dt * drho
    return State(x, st.v.copy(), rho_new, drho, st.m, st.t)


def acoustic_substep(st: State, w: Walls, nb, acc_prior, dt: float, prm: Params, geometry=None):
    """One pressure relaxation followed by one density relaxation with step dt."""
    half, dvdt = pressure_relaxation(st, w, nb, acc_prior, dt, prm, geometry)
    out = density_relaxation(half, w, nb, dt, prm, geometry)
    out.t = st.t + dt
    return out, dvdt, half


@dataclass
class StepInfo:
    dt_ad: float
    substeps: int
    dts: list = field(default_factory=list)
    pairs: int = 0


def advection_step(st: State, w: Walls, prm: Params, neighbours=neighbour_sets, frozen=False):
    """One dual-criteria step: neighbour set, Dt_ad, density re-initialisation, viscous
    acceleration, then acoustic substeps until Dt_ad is covered (Sec. 2.3-2.4, R7).
    frozen=True keeps the pair geometry of the configuration update (reading R11)."""
    st = st.copy()
    nb = neighbours(st.x, w.x, prm)
    Dt = dt_advection(st.v, prm)
    st.rho = density_summation(st, w, nb, prm)
    acc_prior = viscous_acceleration(st, nb, prm)
    geometry = frozen_geometry(st, w, nb, prm) if frozen else None
    tau = 0.0
    info = StepInfo(dt_ad=Dt, substeps=0, pairs=int(nb[0].size + nb[2].size))
    while tau < Dt * (1.0 - LOOP_SLACK):
        dt = min(dt_acoustic(st.v, prm), Dt - tau)
        st, _, _ = acoustic_substep(st, w, nb, acc_prior, dt, prm, geometry)
        tau += dt
        info.substeps += 1
        info.dts.append(dt)
    return st, info


# --------------------------------------------------------------------------------------
# Particle gradients (Eq. gradsph-strong, Eq. gradsph-weak), R18
# --------------------------------------------------------------------------------------
def gradients(st: State, w: Walls, nb, prm: Params) -> dict:
    """Strong- and weak-form SPH gradients of the density and the pressure of every fluid
    particle at the current positions (Sec. 1.1, "particle average and gradient").

    The paper writes both with its grad_i W_ij = e_ij dW/dr, e_ij pointing from i to j,
    which is minus the true gradient of R2. In terms of the true gradient (R18):
      strong  grad f_i = sum_j V_j (f_j - f_i) grad_i W_ij     (f_ij = f_i - f_j, sign absorbed)
      weak    grad f_i = sum_j V_j (f_i + f_j) grad_i W_ij     (-2 sum V_j grad W f~_ij, likewise)
    with V_j = m_j / rho_j for fluid neighbours. A wall neighbour carries the values of the
    one-sided wall problem (R4): p_w = p_i + rho_i g.(r_w - r_i), rho_w from the EoS, V_w its
    volume. Returns {"rho_strong", "rho_weak", "p_strong", "p_weak"}, each (N, d).
    """
    I, J, IW, KW = nb
    N, d = st.x.shape
    p = eos_pressure(st.rho, prm)
    out = {k: np.zeros((N, d)) for k in ("rho_strong", "rho_weak", "p_strong", "p_weak")}
    if I.size:
        _, r, e = _geometry(st.x[I], st.x[J], prm)
        grad = (-e) * kernel_dW(r, prm.h, prm.dim)[:, None]          # true grad_i W_ij (R2)
        Vj = st.m[J] / st.rho[J]
        for f, name in ((st.rho, "rho"), (p, "p")):
            out[name + "_strong"] += _scatter_add(I, (Vj * (f[J] - f[I]))[:, None] * grad, N)
            out[name + "_weak"] += _scatter_add(I, (Vj * (f[I] + f[J]))[:, None] * grad, N)
    if IW.size:
        rfw, r, e = _geometry(st.x[IW], w.x[KW], prm)
        grad = (-e) * kernel_dW(r, prm.h, prm.dim)[:, None]
        pw = p[IW] + st.rho[IW] * ((-rfw) @ prm.gravity)
        rhow = prm.rho0 + pw / prm.c0 ** 2
        Vw = w.V[KW]
        for fi, fw, name in ((st.rho[IW], rhow, "rho"), (p[IW], pw, "p")):
            out[name + "_strong"] += _scatter_add(IW, (Vw * (fw - fi))[:, None] * grad, N)
            out[name + "_weak"] += _scatter_add(IW, (Vw * (fi + fw))[:, None] * grad, N)
    return out


# --------------------------------------------------------------------------------------
# FP64 diagnostics
# --------------------------------------------------------------------------------------
def diagnostics(st: State, prm: Params) -> dict:
    """Conservation and bulk quantities: mass, momentum, kinetic, potential (reference
    at the origin: -m g.r) and internal energy of the EoS (c0^2 (ln(rho/rho0) + rho0/rho - 1)
    per unit mass), density deviation, front position (max x), time."""
    m = st.m
    ke = 0.5 * np.sum(m * np.sum(st.v * st.v, axis=1))
    pe = -np.sum(m * (st.x @ prm.gravity))
    ratio = st.rho / prm.rho0
    ie = np.sum(m * prm.c0 ** 2 * (np.log(ratio) + 1.0 / ratio - 1.0))
    dev = np.abs(ratio - 1.0)
    return {
        "mass": float(np.sum(m)),
        "momentum": np.sum(m[:, None] * st.v, axis=0),
        "kinetic": float(ke),
        "potential": float(pe),
        "internal": float(ie),
        "energy": float(ke + pe + ie),
        "max_rho_dev": float(dev.max()) if dev.size else 0.0,
        "mean_rho_dev": float(dev.mean()) if dev.size else 0.0,
        "front_x": float(st.x[:, 0].max()) if st.x.size else 0.0,
        "t": float(st.t),
    }


def run(problem, t_end: float | None = None, n_advection: int | None = None,
        record_every: int = 1, callback=None):
    """Integrate a problem until t_end (or for n_advection steps); returns (state, series)."""
    prm = Params.from_problem(problem)
    st, w = state_from_problem(problem)
    t_end = problem.t_end if (t_end is None and n_advection is None) else t_end
    series = [diagnostics(st, prm) | {"substeps": 0}]
    k = 0
    total_sub = 0
    while True:
        if n_advection is not None and k >= n_advection:
            break
        if t_end is not None and st.t >= t_end * (1.0 - LOOP_SLACK):
            break
        st, info = advection_step(st, w, prm)
        k += 1
        total_sub += info.substeps
        if k % record_every == 0:
            series.append(diagnostics(st, prm) | {"substeps": total_sub})
        if callback is not None:
            callback(k, st, info)
    return st, series
