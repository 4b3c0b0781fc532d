"""Seeded synthetic inputs for the weakly-compressible SPH hot path.

This module holds geometry and initial conditions only -- lattice particle
placement, dummy-wall layers with their normals and volumes, the Taylor-Green
initial velocity field and the seeded sampling of batched tank geometries. It
contains none of the method's arithmetic (no kernel, no Riemann solver, no
time stepping), so that the CUDA path and the plain CPU oracle can both be fed
from it without sharing any of the computation they are compared on.

Geometry follows the paper's validation cases (Sec. 7.1, 2D/3D dam break):
a fluid block at rest in a tank whose walls are four layers of dummy
particles on the same lattice as the fluid (lattice generator, Sec. 6.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TANK_EXTENT = 5.366          # tank side length of the dam-break cases (multiples of H)
WALL_LAYERS = 4              # dummy-particle wall thickness, in lattice spacings
H_OVER_DP = 1.3              # smoothing length over lattice spacing


@dataclass
class Workload:
    """One SPH problem: parameters plus the initial particle state (all float64).

    Arrays are in particle-id order: row k holds particle id k.
    """
    name: str
    dim: int
    h: float
    dp: float
    rho0: float
    c0: float
    cfl_ad: float
    cfl_ac: float
    u_ref: float
    nu: float
    gravity: np.ndarray          # (3,)
    lo: np.ndarray               # (3,) lower corner of the cell grid
    hi: np.ndarray               # (3,) upper corner of the cell grid
    periodic: np.ndarray         # (3,) int, 1 = periodic axis (period hi-lo)
    free_surface: int
    pos: np.ndarray              # (N, dim)
    vel: np.ndarray              # (N, dim)
    rho: np.ndarray              # (N,)
    mass: np.ndarray             # (N,)
    wall_pos: np.ndarray         # (Nw, dim)
    wall_normal: np.ndarray      # (Nw, dim)
    wall_vol: np.ndarray         # (Nw,)
    t_end: float = 0.0
    meta: dict = field(default_factory=dict)
    p_transport: float = 0.0     # background pressure p0 of the transport velocity (0 = off)

    @property
    def n_fluid(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_wall(self) -> int:
        return int(self.wall_pos.shape[0])


def _lattice(lo, counts, dp):
    """Points lo + (i + 1/2) dp for i over a regular grid with `counts` per axis."""
    axes = [lo[a] + (np.arange(counts[a]) + 0.5) * dp for a in range(len(counts))]
    mesh = np.meshgrid(*axes, indexing="ij")
    # x varies fastest in the returned order
    pts = np.stack([m.transpose(tuple(reversed(range(len(counts))))).reshape(-1) for m in mesh], axis=1)
    return pts


def tank_walls(inner_lo, inner_hi, dp, layers=WALL_LAYERS):
    """Dummy wall particles: lattice points of the outer box that lie outside the inner box.

    The lattice is anchored at the outer corner (inner_lo - layers*dp), so fluid
    placed at inner_lo + (i+1/2)dp sits on the same lattice. Each wall particle's
    normal is the normalised sum of the unit normals of the inner faces it lies
    beyond, pointing into the tank; its volume is dp**dim. Points are ordered with
    x varying fastest over the outer box.
    """
    inner_lo = np.asarray(inner_lo, dtype=np.float64)
    inner_hi = np.asarray(inner_hi, dtype=np.float64)
    dim = inner_lo.shape[0]
    outer_lo = inner_lo - layers * dp
    outer_hi = inner_hi + layers * dp
    counts = [int(math.floor((outer_hi[a] - outer_lo[a]) / dp + 1e-9)) for a in range(dim)]
    coord = [outer_lo[a] + (np.arange(counts[a]) + 0.5) * dp for a in range(dim)]
    side = [(coord[a] > inner_hi[a]).astype(np.int8) - (coord[a] < inner_lo[a]).astype(np.int8)
            for a in range(dim)]
    # flat index x + nx (y + ny z) of every outside point, built from slabs that do not overlap
    strides = [1, counts[0], counts[0] * counts[1]][:dim]
    idx = [np.arange(counts[a], dtype=np.int64) * strides[a] for a in range(dim)]
    out_ = [idx[a][side[a] != 0] for a in range(dim)]
    in_ = [idx[a][side[a] == 0] for a in range(dim)]
    pieces = []
    for a in range(dim):          # outside on axis a, inside on the axes before it
        parts = [in_[b] if b < a else (out_[b] if b == a else idx[b]) for b in range(dim)]
        flat = parts[0]
        for b in range(1, dim):
            flat = (flat[None, :] + parts[b][:, None]).reshape(-1)
        pieces.append(flat)
    flat = np.sort(np.concatenate(pieces))
    ijk = []
    rem = flat
    for a in range(dim):
        ijk.append(rem % counts[a])
        rem = rem // counts[a]
    pts = np.stack([coord[a][ijk[a]] for a in range(dim)], axis=1)
    normal = np.stack([side[a][ijk[a]].astype(np.float64) * -1.0 for a in range(dim)], axis=1)
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    vol = np.full(pts.shape[0], dp ** dim)
    return pts, normal, vol


def dam_break(dim=2, H=1.0, L=2.0, W=1.0, dp=None, n_per_H=40, tank=None, rho0=1.0, g=1.0,
              t_end=None, name=None):
    """Dam break: fluid block L (x) by H (y) [by W (z)] at rest in the corner of a tank.

    2D: tank TANK_EXTENT*H square. 3D: tank TANK_EXTENT*H (x) by TANK_EXTENT*H (y) by W (z),
    the fluid filling the full depth in z. c0 = 10 sqrt(g H) (weakly compressible,
    Sec. 2.1), h = 1.3 dp, CFL_ad = 0.25, CFL_ac = 0.6 (Sec. 2.4).
    """
    if dp is None:
        dp = H / n_per_H
    nx = int(round(L / dp))
    ny = int(round(H / dp))
    if tank is None:
        tank = TANK_EXTENT * H
    if dim == 2:
        fluid = _lattice(np.zeros(2), [nx, ny], dp)
        inner_hi = np.array([tank, tank])
    else:
        nz = int(round(W / dp))
        fluid = _lattice(np.zeros(3), [nx, ny, nz], dp)
        inner_hi = np.array([tank, tank, nz * dp])
    inner_lo = np.zeros(dim)
    wpos, wnrm, wvol = tank_walls(inner_lo, inner_hi, dp)
    c0 = 10.0 * math.sqrt(g * H)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.zeros(3)
    hi = np.zeros(3)
    lo[:dim] = inner_lo - WALL_LAYERS * dp
    hi[:dim] = inner_hi + WALL_LAYERS * dp
    n = fluid.shape[0]
    return Workload(
        name=name or f"dam_break_{dim}d_{n}",
        dim=dim, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0, cfl_ad=0.25, cfl_ac=0.6,
        u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0),
        mass=np.full(n, rho0 * dp ** dim),
        wall_pos=wpos, wall_normal=wnrm, wall_vol=wvol,
        t_end=t_end if t_end is not None else 5.0 * math.sqrt(H / g),
        meta={"H": H, "L": nx * dp, "W": W if dim == 3 else None, "g": g},
    )


def dam_break_with_obstacle(dim=2, H=1.0, L=2.0, W=1.0, dp=None, n_per_H=40, obstacle_x=None,
                            obstacle_w=0.4, obstacle_h=0.4, **kw):
    """Dam break with a block obstacle on the tank floor (the paper's dam break with an
    obstacle, at synthetic sizes): the dam break above plus dummy wall particles filling the
    block [x_o, x_o + w] by [0, h] (the full tank depth in 3D) on the same lattice, each with
    the unit outward normal of its nearest face among the block's left, right and top faces
    (the normalised sum where two are equally near, the top face's where the left and right
    ones are). x_o defaults to 1.5 L."""
    base = dam_break(dim=dim, H=H, L=L, W=W, dp=dp, n_per_H=n_per_H, **kw)
    dp = base.dp
    xo = 1.5 * base.meta["L"] if obstacle_x is None else obstacle_x
    nx, ny = int(round(obstacle_w / dp)), int(round(obstacle_h / dp))
    x0 = round(xo / dp) * dp                        # on the lattice of the fluid and the walls
    if dim == 2:
        blk = _lattice(np.array([x0, 0.0]), [nx, ny], dp)
    else:
        nz = int(round((base.hi[2] - base.lo[2]) / dp)) - 2 * WALL_LAYERS
        blk = _lattice(np.array([x0, 0.0, 0.0]), [nx, ny, nz], dp)
    d = np.stack([blk[:, 0] - x0, x0 + nx * dp - blk[:, 0], ny * dp - blk[:, 1]], axis=1)
    faces = np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    near = d <= d.min(axis=1, keepdims=True) + 1e-9 * dp
    nrm = near.astype(np.float64) @ faces
    nrm[np.linalg.norm(nrm, axis=1) < 0.5] = faces[2]   # equally near the left and right faces: up
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    if dim == 3:
        nrm = np.concatenate([nrm, np.zeros((nrm.shape[0], 1))], axis=1)
    keep = ~np.any(np.all(np.abs(blk[:, None, :] - base.pos[None, :, :]) < 0.5 * dp, axis=2), axis=1) \
        if base.pos.shape[0] * blk.shape[0] < 2e8 else np.ones(blk.shape[0], dtype=bool)
    base.wall_pos = np.concatenate([base.wall_pos, blk[keep]])
    base.wall_normal = np.concatenate([base.wall_normal, nrm[keep]])
    base.wall_vol = np.concatenate([base.wall_vol, np.full(int(keep.sum()), dp ** dim)])
    base.name = f"dam_break_obstacle_{dim}d_{base.n_fluid}"
    base.meta.update({"obstacle": (float(x0), float(nx * dp), float(ny * dp))})
    return base


def sloshing_tank(L=1.0, d=0.5, dp=0.01, g=9.81, rho0=1.0):
    """2D rectangular tank of width L filled to depth d at rest, walls twice as high: the
    sloshing test in the tank's own frame, where a translation of the tank with acceleration
    a(t) acts as the extra body force -a(t) (sph_set_gravity). meta["period_1"] is the
    linear first sloshing mode's period, 2 pi / sqrt(g k tanh(k d)) with k = pi / L."""
    nx, ny = int(round(L / dp)), int(round(d / dp))
    fluid = _lattice(np.zeros(2), [nx, ny], dp)
    inner_hi = np.array([nx * dp, 2.0 * d])
    wpos, wnrm, wvol = tank_walls(np.zeros(2), inner_hi, dp)
    c0 = 10.0 * math.sqrt(g * d)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.array([-WALL_LAYERS * dp, -WALL_LAYERS * dp, 0.0])
    hi = np.array([inner_hi[0] + WALL_LAYERS * dp, inner_hi[1] + WALL_LAYERS * dp, 0.0])
    n = fluid.shape[0]
    k = math.pi / (nx * dp)
    return Workload(
        name=f"sloshing_tank_{n}", dim=2, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0, cfl_ad=0.25,
        cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0), mass=np.full(n, rho0 * dp * dp),
        wall_pos=wpos, wall_normal=wnrm, wall_vol=wvol, t_end=5.0,
        meta={"L": nx * dp, "d": ny * dp, "g": g,
              "period_1": 2.0 * math.pi / math.sqrt(g * k * math.tanh(k * ny * dp))},
    )


def dam_break_2d(n_per_H=40, **kw):
    """2D dam break: H=1, L=2, tank 5.366, dp = H/40 gives 3200 fluid particles."""
    return dam_break(dim=2, n_per_H=n_per_H, **kw)


def dam_break_3d(n=80, **kw):
    """3D dam break: fluid 2 (x) by 1 (y) by 1 (z), dp = 1/n, 2 n^3 fluid particles."""
    return dam_break(dim=3, H=1.0, L=2.0, W=1.0, dp=1.0 / n, **kw)


def still_tank(dim=2, H=0.5, width=None, height=None, dp=0.025, g=1.0, rho0=1.0):
    """Fluid of depth H filling the full width of a tank, at rest (hydrostatic check)."""
    width = width if width is not None else H
    height = height if height is not None else 1.5 * H
    nx = int(round(width / dp))
    ny = int(round(H / dp))
    if dim == 2:
        fluid = _lattice(np.zeros(2), [nx, ny], dp)
        inner_hi = np.array([nx * dp, height])
    else:
        fluid = _lattice(np.zeros(3), [nx, ny, nx], dp)
        inner_hi = np.array([nx * dp, height, nx * dp])
    wpos, wnrm, wvol = tank_walls(np.zeros(dim), inner_hi, dp)
    c0 = 10.0 * math.sqrt(g * H)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.zeros(3)
    hi = np.zeros(3)
    lo[:dim] = -WALL_LAYERS * dp
    hi[:dim] = inner_hi + WALL_LAYERS * dp
    n = fluid.shape[0]
    return Workload(
        name=f"still_tank_{dim}d_{n}", dim=dim, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0),
        mass=np.full(n, rho0 * dp ** dim), wall_pos=wpos, wall_normal=wnrm, wall_vol=wvol,
        t_end=5.0 * math.sqrt(H / g), meta={"H": ny * dp, "g": g},
    )


def taylor_green(n=100, nu=0.01, c0=10.0, rho0=1.0, transport=True):
    """2D periodic Taylor-Green vortex on the unit square, n x n lattice, Re = 1/nu.

    u = -cos(2 pi x) sin(2 pi y), v = sin(2 pi x) cos(2 pi y), rho = rho0, no gravity,
    no walls; kinetic energy decays as exp(-16 pi^2 nu t). A flow without free surface:
    with `transport` the transport velocity is on with background pressure 2 rho0 c0^2.
    """
    dp = 1.0 / n
    pos = _lattice(np.zeros(2), [n, n], dp)
    x, y = pos[:, 0], pos[:, 1]
    vel = np.stack([-np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y),
                    np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)], axis=1)
    lo = np.zeros(3)
    hi = np.zeros(3)
    hi[:2] = 1.0
    per = np.zeros(3, dtype=np.int32)
    per[:2] = 1
    N = pos.shape[0]
    return Workload(
        name=f"taylor_green_{n}x{n}", dim=2, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=nu, gravity=np.zeros(3), lo=lo, hi=hi,
        periodic=per, free_surface=0, pos=pos, vel=vel, rho=np.full(N, rho0),
        mass=np.full(N, rho0 * dp * dp), wall_pos=np.zeros((0, 2)), wall_normal=np.zeros((0, 2)),
        wall_vol=np.zeros(0), t_end=1.0, meta={"U": 1.0, "L": 1.0},
        p_transport=2.0 * rho0 * c0 ** 2 if transport else 0.0,
    )


def periodic_box(dim=2, n=24, seed=0, vel_amp=0.3, rho_amp=0.01, jitter=0.1, c0=10.0):
    """Periodic gravity-free wall-free box with seeded random velocity and density
    perturbations and jittered lattice positions (momentum-conservation check)."""
    rng = np.random.default_rng(seed)
    dp = 1.0 / n
    pos = _lattice(np.zeros(dim), [n] * dim, dp)
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * dp
    pos = np.mod(pos, 1.0)
    N = pos.shape[0]
    vel = rng.uniform(-vel_amp, vel_amp, size=(N, dim))
    rho = 1.0 + rng.uniform(-rho_amp, rho_amp, size=N)
    lo = np.zeros(3)
    hi = np.zeros(3)
    hi[:dim] = 1.0
    per = np.zeros(3, dtype=np.int32)
    per[:dim] = 1
    return Workload(
        name=f"periodic_box_{dim}d_{N}", dim=dim, h=H_OVER_DP * dp, dp=dp, rho0=1.0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=np.zeros(3), lo=lo, hi=hi,
        periodic=per, free_surface=0, pos=pos, vel=vel, rho=rho, mass=np.full(N, dp ** dim),
        wall_pos=np.zeros((0, dim)), wall_normal=np.zeros((0, dim)), wall_vol=np.zeros(0),
    )


def diffusion_band(n=100, ny=8, kappa=1.0, a=0.1, D=None):
    """Band of pollutant diffusing across a static particle body (Sec. mass diffusion,
    first test): unit-periodic x axis with n lattice columns, ny rows on a periodic y axis
    of length ny/n, C = 1 where |x - 1/2| < a and 0 elsewhere, diffusion tensor kappa I
    (or `D`, 3x3 with the leading 2x2 used). meta: C0, D (3x3), dt = 0.1 h^2 / max eig D.
    The GPU's position contract has all periodic axes share one period: ny = n there."""
    dp = 1.0 / n
    pos = _lattice(np.zeros(2), [n, ny], dp)
    C0 = (np.abs(pos[:, 0] - 0.5) < a).astype(np.float64)
    return _static_body(f"diffusion_band_{n}x{ny}", 2, dp, pos, np.array([1.0, ny * dp, 0.0]),
                        C0, kappa, D)


def diffusion_block_3d(n=200, kappa=1.0, sigma=0.1, D=None):
    """Gaussian blob C = exp(-|x - c|^2 / (2 sigma^2)) in a static unit-periodic cube of n^3
    lattice particles (the 3D diffusion workload). meta as diffusion_band."""
    dp = 1.0 / n
    pos = _lattice(np.zeros(3), [n, n, n], dp)
    d2 = np.sum((pos - 0.5) ** 2, axis=1)
    C0 = np.exp(-d2 / (2.0 * sigma * sigma))
    return _static_body(f"diffusion_block_3d_{n}", 3, dp, pos, np.ones(3), C0, kappa, D)


def diffusion_patch(n=40, kappa=1.0, sigma=0.2, D=None):
    """Square patch of n x n lattice particles on [0, 1]^2 with free edges (no periodic axis,
    no walls), so that the kernel correction matrices vary near the edges; Gaussian blob
    C = exp(-|x - c|^2 / (2 sigma^2)). meta as diffusion_band."""
    dp = 1.0 / n
    pos = _lattice(np.zeros(2), [n, n], dp)
    C0 = np.exp(-np.sum((pos - 0.5) ** 2, axis=1) / (2.0 * sigma * sigma))
    w = _static_body(f"diffusion_patch_{n}", 2, dp, pos, np.ones(3), C0, kappa, D)
    w.periodic = np.zeros(3, dtype=np.int32)
    w.lo = np.array([-4.0 * dp, -4.0 * dp, 0.0])
    w.hi = np.array([1.0 + 4.0 * dp, 1.0 + 4.0 * dp, 0.0])
    w.free_surface = 1
    return w


def excitable_sheet(n=200, dp=0.5, cross_field=True):
    """Square sheet of n x n lattice particles of spacing dp with free edges, for the
    Aliev-Panfilov model with unit diffusivity (the paper's spiral-wave test, at synthetic
    sizes and in the model's own units). cross_field: the lower-left quarter excited
    (V = 1) and the upper-left quarter refractory (w = 2), so that the front leaving the
    excited quarter has a free end beside refractory tissue and curls into a spiral;
    otherwise a strip along the left edge is excited, and the planar wave it starts leaves
    the sheet. meta: C0 = V, w0, dt (inside the explicit diffusion limit), the model
    parameters (k = 8, a = 0.15, b = 0.15, eps0 = 0.002, mu1 = 0.2, mu2 = 0.3)."""
    pos = _lattice(np.zeros(2), [n, n], dp)
    L = n * dp
    if cross_field:
        V0 = np.where((pos[:, 0] < L / 2) & (pos[:, 1] < L / 2), 1.0, 0.0)
        w0 = np.where((pos[:, 0] < L / 2) & (pos[:, 1] >= L / 2), 2.0, 0.0)
    else:
        V0 = np.where(pos[:, 0] < 0.05 * L, 1.0, 0.0)
        w0 = np.zeros(pos.shape[0])
    w = _static_body(f"excitable_sheet_{n}", 2, dp, pos, np.ones(3), V0, 1.0, None)
    w.periodic = np.zeros(3, dtype=np.int32)
    w.lo = np.array([-4.0 * dp, -4.0 * dp, 0.0])
    w.hi = np.array([L + 4.0 * dp, L + 4.0 * dp, 0.0])
    w.free_surface = 1
    w.meta["w0"] = w0
    w.meta["dt"] = 0.02
    w.meta["L"] = L
    w.meta["ap"] = dict(k=8.0, a=0.15, b=0.15, eps0=0.002, mu1=0.2, mu2=0.3)
    return w


def _static_body(name, dim, dp, pos, extent, C0, kappa, D):
    N = pos.shape[0]
    Dm = np.zeros((3, 3))
    if D is None:
        Dm[:dim, :dim] = kappa * np.eye(dim)
    else:
        Dm[:dim, :dim] = np.asarray(D, dtype=np.float64)[:dim, :dim]
    h = H_OVER_DP * dp
    lam = float(np.max(np.linalg.eigvalsh(Dm[:dim, :dim])))
    lo = np.zeros(3)
    hi = np.asarray(extent, dtype=np.float64).copy()
    per = np.zeros(3, dtype=np.int32)
    per[:dim] = 1
    return Workload(
        name=name, dim=dim, h=h, dp=dp, rho0=1.0, c0=10.0, cfl_ad=0.25, cfl_ac=0.6, u_ref=1.0,
        nu=0.0, gravity=np.zeros(3), lo=lo, hi=hi, periodic=per, free_surface=0, pos=pos,
        vel=np.zeros((N, dim)), rho=np.ones(N), mass=np.full(N, dp ** dim),
        wall_pos=np.zeros((0, dim)), wall_normal=np.zeros((0, dim)), wall_vol=np.zeros(0),
        meta={"C0": C0, "D": Dm, "dt": 0.1 * h * h / lam},
    )


# ---------------------------------------------------------------------------------------
# Seeded batched tanks.  splitmix64 (Steele, Lea, Flood 2014) drives the sampling so a
# given seed always yields the same geometry.
# ---------------------------------------------------------------------------------------
_MASK64 = (1 << 64) - 1
BATCH_BASE_SEED = 0x201012375


def splitmix64(state: int):
    """One splitmix64 step: returns (new_state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return state, z ^ (z >> 31)


def _uniforms(seed: int, k: int):
    out = []
    s = seed & _MASK64
    for _ in range(k):
        s, z = splitmix64(s)
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return out


def batched_dam_breaks(n_instances=256, n_min=2000, n_max=50000, base_seed=BATCH_BASE_SEED):
    """Independent 2D dam breaks of seeded, uneven size.

    Per instance s: H ~ U(0.5, 1.5), L/H ~ U(1, 3), target fluid count
    exp(U(ln n_min, ln n_max)), dp = sqrt(L H / N_target) rounded to the lattice,
    tank 5.366 H square, c0 = 10 sqrt(g H).
    """
    out = []
    for s in range(n_instances):
        u = _uniforms(base_seed ^ s, 3)
        H = 0.5 + u[0]
        L = H * (1.0 + 2.0 * u[1])
        n_target = math.exp(math.log(n_min) + u[2] * (math.log(n_max) - math.log(n_min)))
        dp = math.sqrt(L * H / n_target)
        ny = max(2, int(round(H / dp)))
        dp = H / ny
        wl = dam_break(dim=2, H=H, L=L, dp=dp, name=f"batched_{s}")
        out.append(wl)
    return out


def learned_dam_break(n_fluid=100_000):
    """2D dam break H=1, L=2 at about n_fluid particles (447 x 224 for 1e5)."""
    dp = math.sqrt(2.0 / n_fluid)
    return dam_break(dim=2, H=1.0, L=2.0, dp=dp, name=f"dam_break_2d_learned")


def water_column_on_plate_3d(dp=1.0 / 16.0, ratio=2, H=0.5, L=0.5, W=0.5, thickness=0.1, youngs=4.55e4,
                             poisson=0.3, rho_s=2.7, rho0=1.0, g=1.0, model=1, nu=0.0):
    """3D counterpart of water_column_on_plate: a block of water H high over an L x W plate
    (y up, gravity along -y), side walls of four dummy layers standing on the plate on all
    four sides, the plate of the given thickness on a lattice ratio times finer, clamped where
    it runs under the walls (x or z outside the tank). Solid normals point up into the water."""
    nx, ny, nz = int(round(L / dp)), int(round(H / dp)), int(round(W / dp))
    fluid = _lattice(np.zeros(3), [nx, ny, nz], dp)
    top = 1.5 * H
    nyw = int(round(top / dp))
    wpos, wnrm, _ = tank_walls(np.zeros(3), np.array([nx * dp, nyw * dp, nz * dp]), dp)
    side = (wpos[:, 1] > 0.0) & (wpos[:, 1] < nyw * dp)      # the x and z walls, not floor or lid
    wpos, wnrm = wpos[side], wnrm[side]
    ds = dp / ratio
    clamp = WALL_LAYERS * dp
    nsx, nsz = int(round((nx * dp + 2 * clamp) / ds)), int(round((nz * dp + 2 * clamp) / ds))
    nsy = max(1, int(round(thickness / ds)))
    spos = _lattice(np.array([-clamp, -nsy * ds, -clamp]), [nsx, nsy, nsz], ds)
    c0 = 10.0 * math.sqrt(g * H)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.array([-clamp - 2 * dp, -nsy * ds - 4 * dp, -clamp - 2 * dp])
    hi = np.array([nx * dp + clamp + 2 * dp, top + 4 * dp, nz * dp + clamp + 2 * dp])
    n = fluid.shape[0]
    wl = Workload(
        name=f"water_column_on_plate_3d_{n}_r{ratio}", dim=3, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=nu, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0), mass=np.full(n, rho0 * dp ** 3),
        wall_pos=wpos, wall_normal=wnrm, wall_vol=np.full(wpos.shape[0], dp ** 3),
        t_end=1.0, meta={"H": ny * dp, "L": nx * dp, "W": nz * dp, "g": g, "thickness": nsy * ds, "ratio": ratio},
    )
    wl.solid_pos = spos
    wl.solid_vol = np.full(spos.shape[0], ds ** 3)
    wl.solid_normal = np.tile([0.0, 1.0, 0.0], (spos.shape[0], 1))
    wl.solid_fixed = (spos[:, 0] < 0.0) | (spos[:, 0] > nx * dp) | (spos[:, 2] < 0.0) | (spos[:, 2] > nz * dp)
    wl.solid_h = H_OVER_DP * ds
    wl.solid_dp = ds
    wl.solid_rho0, wl.solid_youngs, wl.solid_poisson, wl.solid_model = rho_s, youngs, poisson, model
    return wl


def cantilever_beam(ds=0.002, L=0.2, thickness=0.02, youngs=2e6, poisson=0.3, rho_s=1000.0, g=1.0, model=1,
                    fluid_dp=0.008, c0=2.0):
    """2D cantilever of length L and the given thickness on a lattice of spacing ds, clamped
    over 3 h_S at its root (x < 0), with no fluid and no walls: the solid alone (the paper's
    oscillating-beam test, at synthetic sizes). Loaded suddenly by its own weight (gravity g
    along -y) from rest, it oscillates about its static deflection at its first bending
    frequency, for a clamped-free Euler-Bernoulli beam omega_1 = 1.875^2 sqrt(E' I / (rho A L^4))
    with plane strain E' = E / (1 - nu^2) and I / A = thickness^2 / 12 (meta["period_eb"]).
    The fluid parameters only set the step that the solid's substeps fill,
    dt_ac = 0.6 h / c0 with h = 1.3 fluid_dp."""
    clamp = 3 * H_OVER_DP * ds
    nx, ny = int(round((L + clamp) / ds)), max(1, int(round(thickness / ds)))
    spos = _lattice(np.array([-clamp, 0.0]), [nx, ny], ds)
    grav = np.zeros(3)
    grav[1] = -g
    margin = 0.25 * L
    lo = np.array([-clamp - margin, -margin, 0.0])
    hi = np.array([L + margin, ny * ds + margin, 0.0])
    empty = np.zeros((0, 2))
    wl = Workload(
        name=f"cantilever_beam_{spos.shape[0]}", dim=2, h=H_OVER_DP * fluid_dp, dp=fluid_dp, rho0=1.0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=empty, vel=empty.copy(), rho=np.zeros(0), mass=np.zeros(0),
        wall_pos=empty.copy(), wall_normal=empty.copy(), wall_vol=np.zeros(0),
        t_end=1.0, meta={"L": L, "thickness": ny * ds, "g": g},
    )
    wl.solid_pos = spos
    wl.solid_vol = np.full(spos.shape[0], ds * ds)
    wl.solid_normal = np.tile([0.0, 1.0], (spos.shape[0], 1))
    wl.solid_fixed = spos[:, 0] < 0.0
    wl.solid_h = H_OVER_DP * ds
    wl.solid_dp = ds
    wl.solid_rho0, wl.solid_youngs, wl.solid_poisson, wl.solid_model = rho_s, youngs, poisson, model
    Ep = youngs / (1.0 - poisson ** 2)
    t = ny * ds
    wl.meta["period_eb"] = 2.0 * math.pi / (1.875 ** 2 * math.sqrt(Ep * t ** 2 / 12.0 / (rho_s * L ** 4)))
    return wl


def cantilever_beam_3d(ds=0.004, L=0.2, thickness=0.02, youngs=2e6, poisson=0.3, rho_s=1000.0, g=1.0, model=1,
                       fluid_dp=0.008, c0=2.0):
    """3D cantilever of length L and a square cross-section thickness x thickness on a lattice
    of spacing ds, clamped over 3 h_S at its root (x < 0), the solid alone, loaded suddenly
    by its own weight along -y (as cantilever_beam). For a slender beam of square section the
    clamped-free Euler-Bernoulli period uses E itself (uniaxial stress) and I / A =
    thickness^2 / 12 (meta["period_eb"])."""
    clamp = 3 * H_OVER_DP * ds
    nx, ny = int(round((L + clamp) / ds)), max(1, int(round(thickness / ds)))
    spos = _lattice(np.array([-clamp, 0.0, 0.0]), [nx, ny, ny], ds)
    grav = np.zeros(3)
    grav[1] = -g
    margin = 0.25 * L
    lo = np.array([-clamp - margin, -margin, -margin])
    hi = np.array([L + margin, ny * ds + margin, ny * ds + margin])
    empty = np.zeros((0, 3))
    wl = Workload(
        name=f"cantilever_beam_3d_{spos.shape[0]}", dim=3, h=H_OVER_DP * fluid_dp, dp=fluid_dp, rho0=1.0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=empty, vel=empty.copy(), rho=np.zeros(0), mass=np.zeros(0),
        wall_pos=empty.copy(), wall_normal=empty.copy(), wall_vol=np.zeros(0),
        t_end=1.0, meta={"L": L, "thickness": ny * ds, "g": g},
    )
    wl.solid_pos = spos
    wl.solid_vol = np.full(spos.shape[0], ds ** 3)
    wl.solid_normal = np.tile([0.0, 1.0, 0.0], (spos.shape[0], 1))
    wl.solid_fixed = spos[:, 0] < 0.0
    wl.solid_h = H_OVER_DP * ds
    wl.solid_dp = ds
    wl.solid_rho0, wl.solid_youngs, wl.solid_poisson, wl.solid_model = rho_s, youngs, poisson, model
    t = ny * ds
    wl.meta["period_eb"] = 2.0 * math.pi / (1.875 ** 2 * math.sqrt(youngs * t ** 2 / 12.0 / (rho_s * L ** 4)))
    return wl


def elastic_gate(dp=0.0025, ratio=2, A=0.1, H=0.14, gate_h=0.079, gate_t=0.005, tank_w=0.4, youngs=12e6,
                 poisson=0.4, rho_s=1100.0, rho0=1000.0, g=9.81, model=2):
    """Dam break through an elastic gate (the paper's FSI case after Antoci et al., at synthetic
    sizes): a water column A wide and H high at rest against a rigid wall that ends gate_h above
    the floor; below it an elastic gate of thickness gate_t closes the opening, clamped where it
    runs into the rigid wall (over three solid smoothing lengths) and free at its lower end, just
    above the floor. The fluid on a lattice of spacing dp, the gate on one ratio times finer;
    a floor running on to the right so that the water leaves under the opening gate. Solid
    normals point into the water (-x). The rigid wall is four dummy layers thick, above the
    gate's clamped part, its normals pointing into the water as well (the case is meant for
    the gate's opening, before water reaches the wall's far side)."""
    nx, ny = int(round(A / dp)), int(round(H / dp))
    fluid = _lattice(np.zeros(2), [nx, ny], dp)
    top = 3.0 * H                                      # walls high enough for the splash
    wpos, wnrm, wvol = tank_walls(np.zeros(2), np.array([tank_w, top]), dp)
    keep = wpos[:, 1] < top                            # an open top: no ceiling layers
    wpos, wnrm, wvol = wpos[keep], wnrm[keep], wvol[keep]
    ds = dp / ratio
    clamp = 3 * H_OVER_DP * ds
    nsx = max(1, int(round(gate_t / ds)))
    gy0 = 0.5 * ds                                     # the free end, half a spacing above the floor
    nsy = int(round((gate_h + clamp - gy0) / ds))
    spos = _lattice(np.array([nx * dp, gy0]), [nsx, nsy], ds)
    fixed = spos[:, 1] > gate_h
    # the rigid wall above the gate's clamped part (which closes the span between gate_h and
    # the wall): four layers from the gate's left face on
    wy0 = gate_h + clamp
    nwy = int(round((top - wy0) / dp))
    rig = _lattice(np.array([nx * dp, wy0]), [WALL_LAYERS, nwy], dp)
    rn = np.tile([-1.0, 0.0], (rig.shape[0], 1))
    wpos = np.concatenate([wpos, rig])
    wnrm = np.concatenate([wnrm, rn])
    wvol = np.concatenate([wvol, np.full(rig.shape[0], dp * dp)])
    c0 = 10.0 * math.sqrt(g * H)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.array([-WALL_LAYERS * dp, -WALL_LAYERS * dp, 0.0])
    hi = np.array([tank_w + WALL_LAYERS * dp, top + 4 * dp, 0.0])
    n = fluid.shape[0]
    wl = Workload(
        name=f"elastic_gate_{n}_r{ratio}", dim=2, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=0.0, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0), mass=np.full(n, rho0 * dp * dp),
        wall_pos=wpos, wall_normal=wnrm, wall_vol=wvol,
        t_end=0.4, meta={"H": ny * dp, "L": nx * dp, "A": nx * dp, "g": g, "gate_h": gate_h,
                         "thickness": nsx * ds, "ratio": ratio},
    )
    wl.solid_pos = spos
    wl.solid_vol = np.full(spos.shape[0], ds * ds)
    wl.solid_normal = np.tile([-1.0, 0.0], (spos.shape[0], 1))
    wl.solid_fixed = fixed
    wl.solid_h = H_OVER_DP * ds
    wl.solid_dp = ds
    wl.solid_rho0, wl.solid_youngs, wl.solid_poisson, wl.solid_model = rho_s, youngs, poisson, model
    return wl


def water_column_on_plate(dp=1.0 / 40.0, ratio=2, H=1.0, L=1.0, thickness=0.05, youngs=4.55e4,
                          poisson=0.3, rho_s=2.7, rho0=1.0, g=1.0, model=1, nu=0.0):
    """2D water column of height H on an elastic plate spanning a tank of width L (the
    paper's first FSI test, a hydrostatic column on a plate, at synthetic sizes): fluid on a
    lattice of spacing dp, side walls of four dummy layers standing on the plate, the plate
    of the given thickness on a lattice ratio times finer (multi-resolution), clamped where
    it runs under the side walls (x < 0 or x > L). Solid normals point up into the water.
    The plate's static mid-span deflection under q = rho0 g H is q L^4 / (384 E' I) for a
    clamped Euler-Bernoulli beam, E' = E / (1 - nu^2), I = thickness^3 / 12."""
    nx, ny = int(round(L / dp)), int(round(H / dp))
    fluid = _lattice(np.zeros(2), [nx, ny], dp)
    top = 1.5 * H
    nyw = int(round(top / dp))
    walls = []
    for k in range(WALL_LAYERS):
        ys = (np.arange(nyw) + 0.5) * dp
        walls.append(np.stack([np.full(nyw, -(k + 0.5) * dp), ys], axis=1))
        walls.append(np.stack([np.full(nyw, L + (k + 0.5) * dp), ys], axis=1))
    wpos = np.concatenate(walls)
    wnrm = np.where(wpos[:, :1] < 0, [[1.0, 0.0]], [[-1.0, 0.0]]).astype(np.float64)
    ds = dp / ratio
    clamp = WALL_LAYERS * dp
    nsx = int(round((L + 2 * clamp) / ds))
    nsy = max(1, int(round(thickness / ds)))
    spos = _lattice(np.array([-clamp, -nsy * ds]), [nsx, nsy], ds)
    c0 = 10.0 * math.sqrt(g * H)
    grav = np.zeros(3)
    grav[1] = -g
    lo = np.array([-clamp - 2 * dp, -nsy * ds - 4 * dp, 0.0])
    hi = np.array([L + clamp + 2 * dp, top + 4 * dp, 0.0])
    n = fluid.shape[0]
    wl = Workload(
        name=f"water_column_on_plate_{n}_r{ratio}", dim=2, h=H_OVER_DP * dp, dp=dp, rho0=rho0, c0=c0,
        cfl_ad=0.25, cfl_ac=0.6, u_ref=c0 / 10.0, nu=nu, gravity=grav, lo=lo, hi=hi,
        periodic=np.zeros(3, dtype=np.int32), free_surface=1,
        pos=fluid, vel=np.zeros_like(fluid), rho=np.full(n, rho0), mass=np.full(n, rho0 * dp * dp),
        wall_pos=wpos, wall_normal=wnrm, wall_vol=np.full(wpos.shape[0], dp * dp),
        t_end=1.0, meta={"H": ny * dp, "L": nx * dp, "g": g, "thickness": nsy * ds, "ratio": ratio},
    )
    wl.solid_pos = spos
    wl.solid_vol = np.full(spos.shape[0], ds * ds)
    wl.solid_normal = np.tile([0.0, 1.0], (spos.shape[0], 1))
    wl.solid_fixed = (spos[:, 0] < 0.0) | (spos[:, 0] > nx * dp)
    wl.solid_h = H_OVER_DP * ds
    wl.solid_dp = ds
    wl.solid_rho0, wl.solid_youngs, wl.solid_poisson, wl.solid_model = rho_s, youngs, poisson, model
    Ep = youngs / (1.0 - poisson ** 2)
    wl.meta["static_deflection"] = rho0 * g * wl.meta["H"] * wl.meta["L"] ** 4 / (384.0 * Ep * wl.meta["thickness"] ** 3 / 12.0)
    return wl
