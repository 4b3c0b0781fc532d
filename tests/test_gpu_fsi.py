"""GPU parity of the multi-resolution fluid-structure coupling (sph_solid_*) against the FP64
oracle (oracle/fsi.py): a 2D water column on an elastic plate clamped under the side walls,
the plate's lattice two or four times finer than the fluid's.

One coupled acoustic substep from the same representable state: fluid dv/dt, v, rho - rho0
and d rho/dt within 1e-5 relative L2 (the per-substep bar), the solid's kappa equal and its
velocity after the kappa steps within 1e-5; positions are compared through the displacement.
Over a trajectory the plate's mid-span deflection stays within 0.5 % of its extreme.

Also the paper's other solid cases at synthetic sizes: the dam break through an elastic gate
(one substep, and the gate's opening over 0.03 s against the oracle), the cantilever with the
solid alone (its first bending period against the oracle's and the Euler-Bernoulli period,
2D and 3D), and the degenerate cases (a plate beyond the fluid's reach, bad arguments)."""
import copy

import numpy as np
import pytest

from oracle import fsi as f
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import REL_L2_TOL, perturbed_state, rel_l2, representable, walls_representable

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _prepared(ratio, model=f.LINEAR, nu=0.0, thickness=0.05, wl=None):
    if wl is None:
        wl = wk.water_column_on_plate(ratio=ratio, model=model, nu=nu, thickness=thickness)
    wl = copy.copy(wl)
    prm = o.Params.from_problem(wl)
    wl.wall_pos = walls_representable(wl)
    wl.solid_pos = o.dequantise(o.quantise(np.asarray(wl.solid_pos), prm), prm)
    return wl, prm


def _oracle_solid(wl):
    return f.solid_from_problem(wl)


# ratio 8 on a plate 0.1 thick: about 12,000 solid particles, whose constant rows no longer
# fit the solid-step cluster's shared memory next to their state, so the solid steps read
# them from global memory
@pytest.mark.parametrize("ratio,model,nu,thickness", [(2, f.LINEAR, 0.0, 0.05), (4, f.LINEAR, 0.0, 0.05),
                                                      (2, f.NEO_HOOKEAN, 0.01, 0.05), (8, f.LINEAR, 0.0, 0.1)])
def test_one_coupled_substep_matches_the_oracle(sph, ratio, model, nu, thickness):
    wl, prm = _prepared(ratio, model, nu, thickness)
    _coupled_substep_against_oracle(sph, wl, prm, f"ratio {ratio} model {model} nu {nu} thickness {thickness}")


# 3D: a block of water on a plate clamped on four sides. At 0.25 x 0.25 the 1,728 solid
# particles stage their constant rows in the cluster's shared memory, at 0.5 x 0.5 the 3,072
# read them from global memory.
@pytest.mark.parametrize("L,model", [(0.25, f.LINEAR), (0.5, f.NEO_HOOKEAN)])
def test_one_coupled_substep_3d_matches_the_oracle(sph, L, model):
    wl, prm = _prepared(2, wl=wk.water_column_on_plate_3d(L=L, W=L, model=model))
    _coupled_substep_against_oracle(sph, wl, prm, f"3D {L} x {L} model {model}")


def _coupled_substep_against_oracle(sph, wl, prm, label):
    u = np.sqrt(wl.meta["g"] * wl.meta["H"])
    x, v, rho, drho = perturbed_state(wl, 5, 0.2 * u, 0.01)
    st, w = o.state_from_problem(wl)
    st.x = x
    rho = np.maximum(rho, o.density_summation(st, w, o.neighbour_sets(x, w.x, prm), prm)) + 1e-5 * prm.rho0
    xq, v32, rho32, d32 = representable(wl, x, v, rho, drho)
    sim = sph.Simulation(wl, flags=sph.SPH_FLAG_KEEP_ACC)
    sim.set_state(xq, v32, rho32, d32, t=0.0)
    solid = sph.solid_from(sim, wl)
    ns = wl.solid_pos.shape[0]
    sim.build_cells()
    sim.advection_step()
    sim.acoustic_substep()
    acc_gpu = sim.acceleration()
    _, vel_gpu, rho_gpu, drho_gpu = sim.state()
    sg = sph.sph_solid_get_state(sim.handle, solid)
    sph.sph_solid_destroy(solid)
    sim.close()

    st = o.State(xq, v32, rho32, d32, np.asarray(wl.mass, dtype=np.float64), 0.0)
    nb = o.neighbour_sets_quantised(st.x, w.x, prm)
    Dt = o.dt_advection(st.v, prm)
    st.rho = o.density_summation(st, w, nb, prm)
    acc_prior = o.viscous_acceleration(st, nb, prm)
    dt = min(o.dt_acoustic(st.v, prm), Dt)
    sol = _oracle_solid(wl)
    out, dvdt, kappa = f.acoustic_substep(st, w, nb, acc_prior, dt, prm, sol)
    errs = {"dv/dt": rel_l2(acc_gpu, dvdt), "v": rel_l2(vel_gpu, out.v),
            "rho - rho0": rel_l2(rho_gpu - prm.rho0, out.rho - prm.rho0), "drho/dt": rel_l2(drho_gpu, out.drho),
            "solid v": rel_l2(sg["vel"], sol.v), "solid force": rel_l2(sg["force"], sol.f_fluid)}
    print(f"{label}, {ns} solid particles: kappa {kappa} / {sg['solid_steps']}",
          {k: f"{e:.2e}" for k, e in errs.items()})
    assert sg["solid_steps"] == kappa
    for k, e in errs.items():
        assert e < REL_L2_TOL, (k, e)
    _, _, _, dq, _ = o.quantisation(prm)
    disp_g, disp_o = sg["pos"] - wl.solid_pos, sol.x - wl.solid_pos
    assert np.max(np.abs(disp_g - disp_o)) < 2 * kappa * dq + 1e-6 * np.max(np.abs(disp_o))


def test_elastic_gate_substep_matches_the_oracle(sph):
    # the dam break through an elastic gate: a Neo-Hookean gate clamped at its top holds the
    # column from below a rigid wall
    wl, prm = _prepared(2, wl=wk.elastic_gate())
    _coupled_substep_against_oracle(sph, wl, prm, "elastic gate")


def test_elastic_gate_opening_follows_the_oracle():
    # the gate's free end over the first 0.03 s (the water starts to push it open)
    from paper_2010_12375_gb300 import sph as s
    s.load()
    wl, prm = _prepared(2, wl=wk.elastic_gate())
    tip = int(np.argmin(wl.solid_pos[:, 1] - 1e-6 * wl.solid_pos[:, 0]))   # lowest, rightmost
    sim = s.Simulation(wl, flags=s.SPH_FLAG_GRAPH)
    solid = s.solid_from(sim, wl)
    tg, xg = [0.0], [0.0]
    while tg[-1] < 0.03:
        sim.step(1)
        tg.append(sim.diagnostics()["t"])
        xg.append(s.sph_solid_get_state(sim.handle, solid)["pos"][tip, 0] - wl.solid_pos[tip, 0])
    s.sph_solid_destroy(solid)
    sim.close()
    st, w = o.state_from_problem(wl)
    sol = _oracle_solid(wl)
    to, xo = [0.0], [0.0]
    while to[-1] < 0.03:
        st, _, _ = f.advection_step(st, w, prm, sol)
        to.append(st.t)
        xo.append(sol.x[tip, 0] - sol.x0[tip, 0])
    tg, xg, to, xo = map(np.asarray, (tg, xg, to, xo))
    err = np.max(np.abs(xg - np.interp(tg, to, xo))) / np.max(np.abs(xo))
    print(f"gate's free end: opening {xo.max():.3e} at t = {to[-1]:.3f}, GPU vs oracle {err:.2e} of it")
    assert xo.max() > 0.0 and err < 5e-3


def _fluid_above(wl, gap):
    """The workload with only the fluid lying more than `gap` above the plate's top."""
    keep = wl.pos[:, 1] > np.max(wl.solid_pos[:, 1]) + gap
    out = copy.copy(wl)
    out.pos, out.vel, out.rho, out.mass = wl.pos[keep], wl.vel[keep], wl.rho[keep], wl.mass[keep]
    return out


def test_solid_out_of_the_fluids_reach(sph):
    # degenerate coupling: no fluid particle within reach of the plate (the gap is four
    # fluid smoothing lengths, twice the support): no coupling pair anywhere, the plate
    # moves under gravity alone, and the fluid steps exactly as it does without a solid
    wl, prm = _prepared(2)
    wl = _fluid_above(wl, 4 * wl.h)
    _coupled_substep_against_oracle(sph, wl, prm, "fluid out of reach")
    runs = []
    for with_solid in (True, False):
        sim = sph.Simulation(wl, flags=sph.SPH_FLAG_GRAPH)
        solid = sph.solid_from(sim, wl) if with_solid else None
        sim.step(3)
        runs.append(sim.state())
        if with_solid:
            sg = sph.sph_solid_get_state(sim.handle, solid)
            assert np.all(sg["force"] == 0.0) and sg["solid_steps"] > 0
            sph.sph_solid_destroy(solid)
        sim.close()
    for a, b in zip(runs[0], runs[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.slow
def test_plate_deflection_follows_the_oracle():
    pytest.importorskip("scipy")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    wl, prm = _prepared(2)
    sim = s.Simulation(wl, flags=s.SPH_FLAG_GRAPH)
    solid = s.solid_from(sim, wl)
    ns = wl.solid_pos.shape[0]
    mid = int(np.argmin(np.abs(wl.solid_pos[:, 0] - wl.meta["L"] / 2) +
                        np.abs(wl.solid_pos[:, 1] + wl.meta["thickness"] / 2)))
    tg, yg = [0.0], [0.0]
    while tg[-1] < 0.3:
        sim.step(1)
        tg.append(sim.diagnostics()["t"])
        yg.append(s.sph_solid_get_state(sim.handle, solid)["pos"][mid, 1] - wl.solid_pos[mid, 1])
    s.sph_solid_destroy(solid)
    sim.close()
    st, w = o.state_from_problem(wl)
    sol = _oracle_solid(wl)
    to, yo = [0.0], [0.0]
    while to[-1] < 0.3:
        st, _, _ = f.advection_step(st, w, prm, sol)
        to.append(st.t)
        yo.append(sol.x[mid, 1] - sol.x0[mid, 1])
    tg, yg, to, yo = map(np.asarray, (tg, yg, to, yo))
    err = np.max(np.abs(yg - np.interp(tg, to, yo))) / np.max(np.abs(yo))
    print(f"mid-span deflection: extreme {yo.min():.5f}, GPU vs oracle {err:.2e} of it")
    assert err < 5e-3


def _up_crossing_period(ts, ys):
    """Period of an oscillation from the upward crossings of its mean (linear interpolation
    between samples; crossings of one direction only, so an offset of the mean cancels)."""
    ts, ys = np.asarray(ts), np.asarray(ys) - np.mean(ys)
    i = np.nonzero((ys[:-1] < 0.0) & (ys[1:] >= 0.0))[0]
    cr = ts[i] - ys[i] * (ts[i + 1] - ts[i]) / (ys[i + 1] - ys[i])
    return (cr[-1] - cr[0]) / (len(cr) - 1), len(cr)


def _beam_tip_gpu(sph, wl, T):
    """The solid alone, stepped through the library's substep loop (no fluid): tip deflection
    after every fluid substep (each holding kappa solid steps)."""
    sim = sph.Simulation(wl)
    solid = sph.solid_from(sim, wl)
    x0 = wl.solid_pos
    tip = int(np.argmax(x0[:, 0] + 1e-6 * x0[:, 1]))
    t, ts, ys, steps = 0.0, [], [], 0
    while t < T:
        sim.build_cells()
        sim.advection_step()
        done = False
        while not done:
            done, dt = sim.acoustic_substep()
            t += dt
            sg = sph.sph_solid_get_state(sim.handle, solid)
            ts.append(t)
            ys.append(sg["pos"][tip, 1] - x0[tip, 1])
            steps = sg["solid_steps"]                 # solid steps since the solid was attached
    sph.sph_solid_destroy(solid)
    sim.close()
    return np.asarray(ts), np.asarray(ys), steps


def _beam_tip_oracle(wl, T):
    sol = f.solid_from_problem(wl)
    x0 = wl.solid_pos
    tip = int(np.argmax(x0[:, 0] + 1e-6 * x0[:, 1]))
    t, ts, ys = 0.0, [], []
    while t < T:
        dt = 0.8 * f.solid_dt(sol)
        f.solid_step(sol, dt)
        t += dt
        ts.append(t)
        ys.append(sol.x[tip, 1] - x0[tip, 1])
    return np.asarray(ts), np.asarray(ys)


def test_cantilever_oscillates_at_its_first_bending_frequency(sph):
    # the paper's oscillating beam with the solid alone: a cantilever 0.2 long and 0.02 thick
    # loaded suddenly by its weight. At 5 particles across its period matches the oracle's
    # (the same discretisation in FP64); at 10 across it approaches the clamped-free
    # Euler-Bernoulli period from above (the oracle pins the same convergence)
    T = 1.5
    coarse = wk.cantilever_beam(ds=0.004)
    tg, yg, _ = _beam_tip_gpu(sph, coarse, T)
    to, yo = _beam_tip_oracle(coarse, T)
    pg, ng = _up_crossing_period(tg, yg)
    po, no = _up_crossing_period(to, yo)
    fine = wk.cantilever_beam(ds=0.002)
    tf, yf, steps = _beam_tip_gpu(sph, fine, T)
    pf, nf = _up_crossing_period(tf, yf)
    eb = fine.meta["period_eb"]
    print(f"cantilever period: 5 across GPU {pg:.5f} s ({ng} crossings) oracle {po:.5f} s ({no}); "
          f"10 across GPU {pf:.5f} s = {pf / eb:.4f} x Euler-Bernoulli ({eb:.5f} s), {steps} solid steps; "
          f"tip amplitude {np.ptp(yf):.3e} (static deflection x2 {3 * fine.meta['g'] * fine.solid_rho0 * 0.2 ** 4 / (fine.solid_youngs / 0.91 * 0.02 ** 2):.3e})")
    assert ng >= 3 and no >= 3 and nf >= 3
    assert abs(pg / po - 1.0) < 5e-3
    assert 1.0 < pf / eb < 1.09 and abs(pf / eb - 1.0) < abs(pg / eb - 1.0)


def test_3d_cantilever_period_converges_to_euler_bernoulli(sph):
    # a 3D cantilever of square section (5 and 10 particles across, 1,350 and 10,400
    # particles; the finer one reads its constant rows from global memory), loaded by its
    # weight: the first bending period approaches the Euler-Bernoulli period from above
    T = 1.5
    ratios = []
    for ds in (0.004, 0.002):
        wl = wk.cantilever_beam_3d(ds=ds)
        ts, ys, steps = _beam_tip_gpu(sph, wl, T)
        p, n = _up_crossing_period(ts, ys)
        assert n >= 3
        ratios.append(p / wl.meta["period_eb"])
        print(f"3D cantilever, {wl.solid_pos.shape[0]} particles: period {p:.5f} s = {ratios[-1]:.4f} x "
              f"Euler-Bernoulli, {steps} solid steps")
    assert 1.0 < ratios[1] < ratios[0] and ratios[1] < 1.1


def test_solid_refuses_bad_arguments(sph):
    wl, _ = _prepared(2)
    sim = sph.Simulation(wl)
    with pytest.raises(sph.SphError):                      # Poisson ratio out of range
        sph.sph_solid_create(sim.handle, 1, 2.7, 4.5e4, 0.5, wl.solid_h, wl.solid_pos, wl.solid_vol,
                             wl.solid_normal, wl.solid_fixed)
    for count in (0, 16385):                               # particle count outside [1, 16384]
        idx = np.arange(count) % wl.solid_pos.shape[0]
        with pytest.raises(sph.SphError):
            sph.sph_solid_create(sim.handle, 1, 2.7, 4.5e4, 0.3, wl.solid_h, wl.solid_pos[idx], wl.solid_vol[idx],
                                 wl.solid_normal[idx], None if wl.solid_fixed is None else wl.solid_fixed[idx])
    s1 = sph.solid_from(sim, wl)
    with pytest.raises(sph.SphError):                      # one solid per handle
        sph.solid_from(sim, wl)
    sph.sph_solid_destroy(s1)
    sim.close()
    tanks = sph.Simulation(wk.batched_dam_breaks(2, n_min=500, n_max=800))
    with pytest.raises(sph.SphError):                      # single-tank handles only
        sph.solid_from(tanks, wl)
    tanks.close()
