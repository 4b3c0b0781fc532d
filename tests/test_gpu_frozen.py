"""The frozen-geometry reading (R11, SPH_FLAG_FROZEN_GEOMETRY) on the GPU against the
oracle's frozen reading: pair vectors and (dW/dr)/r kept from the configuration update."""
import numpy as np
import pytest

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


def _case(case):
    if case == "dam2d":
        prob, vel_amp, rho_amp = wk.dam_break_2d(), 0.3, 0.01
    elif case == "tg":
        prob, vel_amp, rho_amp = wk.taylor_green(64, transport=False), 0.05, 0.005
    elif case == "dam3d":
        prob, vel_amp, rho_amp = wk.dam_break_3d(16), 0.3, 0.01
    else:
        prob, vel_amp, rho_amp = wk.periodic_box(dim=3, n=12, seed=3), 0.1, 0.01
    prob.wall_pos = walls_representable(prob)
    return prob, vel_amp, rho_amp


def _prepared(prob, vel_amp, rho_amp, seed=11):
    x, v, rho, drho = perturbed_state(prob, seed, vel_amp, rho_amp)
    x = x + np.random.default_rng(seed + 1).uniform(-0.1, 0.1, size=x.shape) * prob.dp
    if np.any(prob.periodic[:prob.dim]):
        x = np.mod(x, 1.0)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    if prm.free_surface:
        # density re-initialisation an identity on both sides: rho* above the sum
        st.x = x
        nb = o.neighbour_sets(x, w.x, prm)
        rho = np.maximum(rho, o.density_summation(st, w, nb, prm)) + 1e-5 * prm.rho0
    return prm, w, representable(prob, x, v, rho, drho)


def test_at_rest_the_first_pressure_relaxation_is_bit_identical(sph):
    # v = 0: no half-step shift, so the frozen table holds exactly what the kernel computes
    prob, _, rho_amp = _case("dam2d")
    prm, w, (xq, v32, rho32, d32) = _prepared(prob, 0.0, rho_amp)
    v32 = np.zeros_like(v32)
    acc = []
    for flags in (sph.SPH_FLAG_KEEP_ACC, sph.SPH_FLAG_KEEP_ACC | sph.SPH_FLAG_FROZEN_GEOMETRY):
        sim = sph.Simulation(prob, flags=flags)
        sim.set_state(xq, v32, rho32, d32, t=0.0)
        sim.build_cells()
        sim.advection_step()
        sim.acoustic_substep()
        acc.append(sim.acceleration())
        sim.close()
    assert np.abs(acc[0] - prm.gravity).max() > 1e-2
    np.testing.assert_array_equal(acc[1], acc[0])


@pytest.mark.parametrize("case", ["dam2d", "tg", "dam3d", "box3d"])
def test_frozen_substeps_match_the_frozen_oracle(sph, case):
    prob, vel_amp, rho_amp = _case(case)
    prm, w, (xq, v32, rho32, d32) = _prepared(prob, vel_amp, rho_amp)
    sim = sph.Simulation(prob, flags=sph.SPH_FLAG_KEEP_ACC | sph.SPH_FLAG_FROZEN_GEOMETRY)
    sim.set_state(xq, v32, rho32, d32, t=0.0)
    sim.build_cells()
    sim.advection_step()
    gpu = []
    for _ in range(3):                      # three substeps on one frozen table
        sim.acoustic_substep()
        gpu.append((sim.acceleration(), *sim.state()))
    sim.close()

    st = o.State(xq, v32, rho32, d32, np.asarray(prob.mass, dtype=np.float64), 0.0)
    nb = o.neighbour_sets_quantised(st.x, w.x, prm)
    Dt = o.dt_advection(st.v, prm)
    st.rho = o.density_summation(st, w, nb, prm)
    acc_prior = o.viscous_acceleration(st, nb, prm)
    geo = o.frozen_geometry(st, w, nb, prm)
    tau = 0.0
    for k in range(3):
        dt = min(o.dt_acoustic(st.v, prm), Dt - tau)
        half, dvdt = o.pressure_relaxation(st, w, nb, acc_prior, dt, prm, geo)
        st = o.density_relaxation(half, w, nb, dt, prm, geo)
        tau += dt
        acc_gpu, pos_gpu, vel_gpu, rho_gpu, _ = gpu[k]
        print(f"{case} substep {k}: rel L2 dv/dt {rel_l2(acc_gpu, dvdt):.2e} v {rel_l2(vel_gpu, st.v):.2e} "
              f"rho - rho0 {rel_l2(rho_gpu - prm.rho0, st.rho - prm.rho0):.2e}")
        assert rel_l2(acc_gpu, dvdt) < REL_L2_TOL
        assert rel_l2(vel_gpu, st.v) < REL_L2_TOL
        # both sides continue from their own states (not re-synchronised between substeps),
        # so the density deviation carries every earlier substep's dt drho/dt error: the
        # per-substep 1e-5 adds up to (k + 1) 1e-5 after substep k
        assert rel_l2(rho_gpu - prm.rho0, st.rho - prm.rho0) < (k + 1) * REL_L2_TOL
        _, _, _, dq, _ = o.quantisation(prm)
        assert np.max(np.abs(o.min_image(pos_gpu - st.x, prm.period))) < 8 * (k + 1) * dq + 1e-7 * prm.dp


def test_frozen_reading_conserves_momentum(sph):
    prob = wk.periodic_box(dim=3, n=16, seed=21, vel_amp=0.3, rho_amp=0.01)
    sim = sph.Simulation(prob, flags=sph.SPH_FLAG_FROZEN_GEOMETRY)
    d0 = sim.diagnostics()
    sim.step(3)
    d1 = sim.diagnostics()
    scale = np.sum(prob.mass[:, None] * np.abs(prob.vel))
    assert np.max(np.abs(d1["momentum"] - d0["momentum"])) < 1e-6 * scale
    assert d1["mass"] == d0["mass"] and d1["substeps"] > d0["substeps"]
    sim.close()


def test_frozen_graph_loop_equals_host_loop(sph):
    prob = wk.dam_break_2d(n_per_H=20)
    a = sph.Simulation(prob, flags=sph.SPH_FLAG_FROZEN_GEOMETRY)
    b = sph.Simulation(prob, flags=sph.SPH_FLAG_FROZEN_GEOMETRY | sph.SPH_FLAG_GRAPH)
    a.step(4)
    b.step(4)
    for u, v in zip(a.state(), b.state()):
        np.testing.assert_array_equal(u, v)
    a.close()
    b.close()


def test_frozen_batched_tanks_match_single_runs(sph):
    # the multi-tank launches (tank constants read per particle) against one tank per handle
    tanks = wk.batched_dam_breaks(n_instances=4, n_min=300, n_max=2000)
    flags = sph.SPH_FLAG_FROZEN_GEOMETRY
    multi = sph.Simulation(tanks, flags=flags)
    multi.step(3)
    pos_m, vel_m, rho_m, _ = multi.state()
    off = multi.fluid_offsets
    for k, t in enumerate(tanks):
        single = sph.Simulation(t, flags=flags)
        single.step(3)
        pos_s, vel_s, rho_s, _ = single.state()
        sl = slice(off[k], off[k + 1])
        np.testing.assert_array_equal(pos_m[sl], pos_s)
        np.testing.assert_array_equal(vel_m[sl], vel_s)
        np.testing.assert_array_equal(rho_m[sl], rho_s)
        single.close()
    multi.close()
