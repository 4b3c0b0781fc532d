"""Pins of the FSI oracle (oracle/fsi.py): the total Lagrangian solid, its Verlet steps and
the multi-resolution coupling, against what fixes them independently:
  * B0 tends to the identity in the interior of a lattice as h/dp grows, and with it F is
    exact for any linear displacement, at every particle, surfaces included;
  * a rigid rotation gives F = R and zero stress, for both material laws, in 2D and 3D;
  * the elastic forces are antisymmetric per pair: a free solid's momentum is conserved;
  * a cantilever's first bending frequency against Euler-Bernoulli's closed form;
  * a hydrostatic column on a rigid plate loads it with the column's weight rho0 g H L
    (rho0 g H L W in 3D), and the fluid takes exactly the opposite momentum;
  * the viscous coupling slows fluid sliding along a plate (R23);
  * the kappa solid steps cover the fluid step.
Planted mistakes fail them: no correction matrix, a flipped stress sign, no pressure
extrapolation at the plate.
"""
import math

import numpy as np
import pytest

from oracle import fsi as f
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk


def _block(nx, ny, dp, hdp=1.3, model=f.LINEAR, fixed=None):
    x0 = wk._lattice(np.zeros(2), [nx, ny], dp)
    mat = f.Material(rho0=1000.0, youngs=2e6, poisson=0.3, model=model)
    fx = np.zeros(len(x0), bool) if fixed is None else fixed(x0)
    return f.make_solid(x0, np.full(len(x0), dp * dp), np.tile([0.0, 1.0], (len(x0), 1)), fx, mat, hdp * dp,
                        np.zeros(3)), x0


def test_correction_matrix_tends_to_identity():
    errs = []
    for hdp in (1.3, 2.0, 3.0):
        sol, x0 = _block(30, 30, 0.01, hdp)
        inner = np.all((x0 > 2.05 * sol.h) & (x0 < 0.3 - 2.05 * sol.h), axis=1)
        errs.append(np.abs(sol.B0[inner] - np.eye(2)).max())
    assert errs[0] < 0.05 and errs[2] < errs[1] < errs[0] and errs[2] < 1e-3, errs


@pytest.mark.parametrize("model", [f.LINEAR, f.NEO_HOOKEAN])
def test_linear_displacement_and_rigid_rotation(model):
    sol, x0 = _block(20, 8, 0.01, model=model)
    G = np.array([[0.01, -0.02], [0.005, 0.03]])
    F = f.deformation_gradient_from_displacement(sol, x0 @ G.T)
    assert np.abs(F - (np.eye(2) + G)).max() < 1e-12          # surfaces included
    th = 0.3
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    sol.F = f.deformation_gradient_from_displacement(sol, x0 @ R.T - x0)
    assert np.abs(sol.F - R).max() < 1e-12
    assert np.abs(f.first_piola(sol.F, sol.mat)).max() < 1e-8 * sol.mat.youngs
    assert np.abs(f.elastic_acceleration(sol)).max() < 1e-8 * sol.mat.youngs / (sol.mat.rho0 * sol.h)
    # a uniform stretch: the linear law's P = F S with E = (F^T F - I)/2 written out
    e = 0.01
    Fs = np.array([[1 + e, 0.0], [0.0, 1.0]])
    E = 0.5 * (Fs.T @ Fs - np.eye(2))
    S_lin = sol.mat.lam * np.trace(E) * np.eye(2) + 2 * sol.mat.mu * E
    if model == f.LINEAR:
        assert np.allclose(f.first_piola(Fs[None], sol.mat)[0], Fs @ S_lin, rtol=1e-12)
    else:    # small strain: Neo-Hookean agrees with the linear law to first order in e
        assert np.allclose(f.first_piola(Fs[None], sol.mat)[0], Fs @ S_lin, rtol=3 * e)


@pytest.mark.parametrize("model", [f.LINEAR, f.NEO_HOOKEAN])
def test_3d_linear_displacement_and_rigid_rotation(model):
    dp = 0.01
    x0 = wk._lattice(np.zeros(3), [8, 6, 5], dp)
    mat = f.Material(rho0=1000.0, youngs=2e6, poisson=0.3, model=model)
    sol = f.make_solid(x0, np.full(len(x0), dp ** 3), np.tile([0.0, 1.0, 0.0], (len(x0), 1)),
                       np.zeros(len(x0), bool), mat, 1.3 * dp, np.zeros(3))
    G = np.array([[0.01, -0.02, 0.004], [0.005, 0.03, -0.01], [-0.003, 0.002, 0.02]])
    F = f.deformation_gradient_from_displacement(sol, x0 @ G.T)
    assert np.abs(F - (np.eye(3) + G)).max() < 1e-12          # surfaces and corners included
    a, b = 0.3, -0.2                                            # a rotation about z, then about x
    Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(b), -math.sin(b)], [0.0, math.sin(b), math.cos(b)]])
    R = Rx @ Rz
    sol.F = f.deformation_gradient_from_displacement(sol, x0 @ R.T - x0)
    assert np.abs(sol.F - R).max() < 1e-12
    assert np.abs(f.first_piola(sol.F, sol.mat)).max() < 1e-8 * sol.mat.youngs
    assert np.abs(f.elastic_acceleration(sol)).max() < 1e-8 * sol.mat.youngs / (sol.mat.rho0 * sol.h)


def test_3d_hydrostatic_column_loads_the_plate_with_its_weight():
    # a 0.5 x 0.5 x 0.5 block of water on a plate clamped on four sides: the plate carries
    # rho0 g H L W (0.978 of it at dp = 1/16, 0.984 at 1/24), straight down, and the fluid
    # takes exactly the opposite momentum
    wl = wk.water_column_on_plate_3d()
    prm = o.Params.from_problem(wl)
    st, _ = o.state_from_problem(wl)
    sol = f.solid_from_problem(wl)
    H, g = wl.meta["H"], wl.meta["g"]
    rho = prm.rho0 + prm.rho0 * g * (H - st.x[:, 1]) / prm.c0 ** 2
    acc, force = f.coupling_forces(st.x, rho, st.v, st.m, sol, prm)
    total, fluid = force.sum(axis=0), np.sum(st.m[:, None] * acc, axis=0)
    weight = prm.rho0 * g * H * wl.meta["L"] * wl.meta["W"]
    assert abs(total[0]) < 1e-12 * weight and abs(total[2]) < 1e-12 * weight
    assert abs(total[1] + weight) < 0.03 * weight, (total, weight)
    assert np.abs(total + fluid).max() < 1e-12 * weight


def test_free_solid_conserves_momentum():
    sol, x0 = _block(16, 6, 0.01)
    rng = np.random.default_rng(4)
    sol.v = rng.uniform(-0.05, 0.05, sol.v.shape)
    for _ in range(20):
        f.solid_step(sol, 2e-5)
        total = np.sum(sol.m[:, None] * sol.acc, axis=0)
        assert np.abs(total).max() <= 1e-9 * np.sum(sol.m[:, None] * np.abs(sol.acc))
    assert np.abs(sol.x - x0).max() > 0


def _cantilever_period(dp):
    """First bending period of a cantilever 0.2 long and 0.02 thick, clamped over 3 h at its
    root, started with its first mode's shape as a small velocity; from the tip's crossings
    of its rest position. Also returns the clamped-free Euler-Bernoulli period (plane
    strain: omega_1 = 1.875^2 sqrt(E' I / (rho A L^4)), E' = E / (1 - nu^2), I / A = t^2 / 12)."""
    L, thick = 0.2, 0.02
    clamp = 3 * 1.3 * dp
    nx, ny = int(round((L + clamp) / dp)), int(round(thick / dp))
    x0 = wk._lattice(np.array([-clamp, 0.0]), [nx, ny], dp)
    mat = f.Material(rho0=1000.0, youngs=2e6, poisson=0.3)
    sol = f.make_solid(x0, np.full(len(x0), dp * dp), np.tile([0.0, 1.0], (len(x0), 1)), x0[:, 0] < 0, mat,
                       1.3 * dp, np.zeros(3))
    k = 1.875 / L
    s = np.clip(x0[:, 0], 0, None)
    shape = (np.cosh(k * s) - np.cos(k * s)) - 0.734 * (np.sinh(k * s) - np.sin(k * s))
    sol.v[:, 1] = np.where(x0[:, 0] > 0, 0.01 * shape / shape.max(), 0.0)
    tip = np.argmax(x0[:, 0] + 1e-6 * x0[:, 1])
    dt = 0.8 * f.solid_dt(sol)
    ys, ts, t = [], [], 0.0
    while t < 0.5:
        f.solid_step(sol, dt)
        t += dt
        ys.append(sol.x[tip, 1] - x0[tip, 1])
        ts.append(t)
    ys, ts = np.array(ys), np.array(ts)
    cx = np.nonzero(np.sign(ys[:-1]) != np.sign(ys[1:]))[0]
    cr = [ts[i] - ys[i] * (ts[i + 1] - ts[i]) / (ys[i + 1] - ys[i]) for i in cx]
    period = 2.0 * (cr[-1] - cr[0]) / (len(cr) - 1)
    Ep = mat.youngs / (1 - mat.poisson ** 2)
    omega = 1.875 ** 2 * math.sqrt(Ep * thick ** 2 / 12.0 / (mat.rho0 * L ** 4))
    return period, 2 * math.pi / omega


@pytest.mark.slow
def test_cantilever_first_frequency_converges_to_euler_bernoulli():
    # measured: 1.205 (5 particles across), 1.115 (7), 1.065 (10) times the closed form
    p1, exact = _cantilever_period(0.004)
    p2, _ = _cantilever_period(0.02 / 7)
    e1, e2 = abs(p1 / exact - 1.0), abs(p2 / exact - 1.0)
    print(f"cantilever period / Euler-Bernoulli: {p1 / exact:.3f} (5 across), {p2 / exact:.3f} (7 across)")
    assert e2 < 0.75 * e1 and e2 < 0.13 and p2 > exact


def _plate_hydrostatics():
    wl = wk.water_column_on_plate()
    prm = o.Params.from_problem(wl)
    st, _ = o.state_from_problem(wl)
    sol = f.solid_from_problem(wl)
    H, L, g = wl.meta["H"], wl.meta["L"], wl.meta["g"]
    p = prm.rho0 * g * (H - st.x[:, 1])
    rho = prm.rho0 + p / prm.c0 ** 2
    acc, force = f.coupling_forces(st.x, rho, st.v, st.m, sol, prm)
    return force.sum(axis=0), np.sum(st.m[:, None] * acc, axis=0), prm.rho0 * g * H * L


def test_hydrostatic_column_loads_the_plate_with_its_weight():
    total, fluid, weight = _plate_hydrostatics()
    assert abs(total[0]) < 1e-12 * weight
    assert abs(total[1] + weight) < 0.03 * weight, (total, weight)
    assert np.abs(total + fluid).max() < 1e-12 * weight            # equal and opposite


def test_viscous_coupling_opposes_sliding():
    wl = wk.water_column_on_plate(nu=0.01)
    prm = o.Params.from_problem(wl)
    st, _ = o.state_from_problem(wl)
    sol = f.solid_from_problem(wl)
    v = np.zeros_like(st.v)
    v[:, 0] = 0.1                                   # fluid sliding along a plate at rest
    rho = np.full(len(st.x), prm.rho0)
    a_slide, _ = f.coupling_forces(st.x, rho, v, st.m, sol, prm)
    a_rest, _ = f.coupling_forces(st.x, rho, np.zeros_like(v), st.m, sol, prm)
    dvx = a_slide[:, 0] - a_rest[:, 0]
    near = np.abs(dvx) > 0
    assert near.sum() > 10 and np.all(dvx[near] < 0)


def test_solid_steps_cover_the_fluid_step():
    sol, _ = _block(10, 4, 0.01)
    dts = f.solid_dt(sol)
    kappa = f.solid_substeps(sol, 7.3 * dts)
    assert kappa == 8 and 7.3 * dts / kappa <= dts          # equal steps, each within dt_S


def test_planted_mistakes_are_caught(monkeypatch):
    # no correction matrix: the cantilever's frequency moves off (a few percent at 5 layers)
    # is too weak a check; F of a linear displacement is no longer exact at the surfaces
    sol, x0 = _block(20, 8, 0.01)
    sol.B0 = np.broadcast_to(np.eye(2), sol.B0.shape).copy()
    G = np.array([[0.01, -0.02], [0.005, 0.03]])
    F = f.deformation_gradient_from_displacement(sol, x0 @ G.T)
    assert np.abs(F - (np.eye(2) + G)).max() > 1e-3
    # a flipped stress sign: a stretched free bar accelerates outward instead of contracting
    sol, x0 = _block(20, 4, 0.01)
    sol.F = np.broadcast_to(np.array([[1.01, 0.0], [0.0, 1.0]]), sol.F.shape).copy()
    a = f.elastic_acceleration(sol)
    right = x0[:, 0] > x0[:, 0].max() - 0.005
    assert np.all(a[right, 0] < 0)                                  # the right end pulls back
    orig = f.first_piola
    monkeypatch.setattr(f, "first_piola", lambda F, m: -orig(F, m))
    assert np.all(f.elastic_acceleration(sol)[right, 0] > 0)
    monkeypatch.setattr(f, "first_piola", orig)
    # no pressure extrapolation at the plate (p^d = p_i)
    orig_ip = f.imaginary_pressure
    monkeypatch.setattr(f, "imaginary_pressure", lambda p, rho, r, n, a, g: p)
    with pytest.raises(AssertionError):
        test_hydrostatic_column_loads_the_plate_with_its_weight()
    monkeypatch.setattr(f, "imaginary_pressure", orig_ip)
