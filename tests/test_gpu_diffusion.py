"""GPU parity of species diffusion (Eq. grad-laplace, two-stage Runge-Kutta) through the C ABI
against the FP64 oracle (oracle/diffusion.py), from identical representable inputs.

Tolerance. The GPU keeps C in FP32 and rounds it after every stage (2 per step), and each
pair term carries a few FP32 roundings, so after k steps
  max |C_gpu - C_oracle| <= 8 k 2^-24 max|C_0| + 1e-5 max|C_oracle - C_0|:
four times the two storage roundings per step, plus a relative error of the accumulated
rates well above FP32's (a sum of 20-80 terms).
"""
import copy
import math

import numpy as np
import pytest

from oracle import diffusion as df
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import representable

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _bound(k, C0, Co):
    return 8 * k * 2.0 ** -24 * np.max(np.abs(C0)) + 1e-5 * np.max(np.abs(Co - C0))


def _representable_problem(prob, mass_jitter=0.0, seed=0):
    p = copy.copy(prob)
    xq, v32, rho32, _ = representable(prob, prob.pos, prob.vel, prob.rho)
    p.pos, p.vel, p.rho = xq, v32, rho32
    m = np.asarray(prob.mass, dtype=np.float64)
    if mass_jitter:
        m = m * np.random.default_rng(seed).uniform(1 - mass_jitter, 1 + mass_jitter, m.shape)
    p.mass = m.astype(np.float32).astype(np.float64)
    return p


def _gpu_run(sph, probs, D, C0, dt, steps, calls=1):
    sim = sph.Simulation(probs)
    try:
        sph.sph_build_cells(sim.handle)
        dim = sim.dim
        sp = sph.sph_species_create(sim.handle, D, dim)
        try:
            sph.sph_species_set(sim.handle, sp, C0)
            for _ in range(calls):
                sph.sph_diffusion_step(sim.handle, sp, dt, steps // calls)
            return sph.sph_species_get(sim.handle, sp, sim.n)
        finally:
            sph.sph_species_destroy(sp)
    finally:
        sim.close()


def _oracle_run(p, D, C0, dt, steps):
    prm = o.Params.from_problem(p)
    return df.run(p.pos, C0, p.mass, p.rho, np.asarray(D)[:p.dim, :p.dim], dt, steps, prm)


def _case(name):
    rng = np.random.default_rng(7)
    if name == "band2d":
        prob = wk.diffusion_band(n=128, ny=128, kappa=1.0, a=0.1)   # periodic axes share one period
        p = _representable_problem(prob)
        C0 = prob.meta["C0"]
        D = prob.meta["D"][:2, :2]
    elif name == "aniso2d":
        p = _representable_problem(wk.periodic_box(2, n=48, seed=3, vel_amp=0.0), mass_jitter=0.1)
        C0 = rng.uniform(0.0, 1.0, p.n_fluid)
        D = np.array([[2.0, 0.6], [0.6, 1.0]])
    elif name in ("iso3d", "aniso3d"):
        p = _representable_problem(wk.periodic_box(3, n=16, seed=5, vel_amp=0.0), mass_jitter=0.1)
        C0 = rng.uniform(-1.0, 1.0, p.n_fluid)
        A = rng.normal(size=(3, 3))
        D = 0.5 * np.eye(3) if name == "iso3d" else A @ A.T + 3.0 * np.eye(3)
    elif name == "walls2d":
        p = _representable_problem(wk.dam_break_2d())
        p.wall_pos = o.dequantise(o.quantise(np.asarray(p.wall_pos), o.Params.from_problem(p)),
                                  o.Params.from_problem(p))
        C0 = rng.uniform(0.0, 1.0, p.n_fluid)
        D = 0.01 * np.eye(2)
    else:
        raise ValueError(name)
    C0 = np.asarray(C0, dtype=np.float32).astype(np.float64)
    dt = 0.1 * p.h ** 2 / float(np.max(np.linalg.eigvalsh(D)))
    return p, D, C0, dt


@pytest.mark.parametrize("name", ["band2d", "aniso2d", "iso3d", "aniso3d", "walls2d"])
def test_diffusion_matches_oracle(sph, name):
    p, D, C0, dt = _case(name)
    steps = 10
    Cg = _gpu_run(sph, p, D, C0, dt, steps)
    Co = _oracle_run(p, D, C0, dt, steps)
    err = np.max(np.abs(Cg - Co))
    assert np.max(np.abs(Co - C0)) > 1e-3            # the species did move
    assert err <= _bound(steps, C0, Co), (name, err, _bound(steps, C0, Co))


def test_diffusion_split_calls_equal_one_call(sph):
    # the species by caller row survives the gather/scatter between calls bit for bit
    p, D, C0, dt = _case("aniso2d")
    a = _gpu_run(sph, p, D, C0, dt, 6, calls=1)
    b = _gpu_run(sph, p, D, C0, dt, 6, calls=3)
    assert np.array_equal(a, b)


def test_species_follows_particles_through_resorting(sph):
    # sph_step moves and re-sorts the fluid; the species stays attached to caller rows,
    # and diffusion on the moved state matches the oracle on that state
    prob = wk.dam_break_2d()
    sim = sph.Simulation(prob)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, 0.01 * np.eye(2), 2)
        C0 = np.random.default_rng(1).uniform(0, 1, sim.n).astype(np.float32).astype(np.float64)
        sph.sph_species_set(sim.handle, sp, C0)
        sph.sph_step(sim.handle, 3)
        assert np.array_equal(sph.sph_species_get(sim.handle, sp, sim.n), C0)
        perm = sph.sph_get_permutation(sim.handle, sim.n)
        assert not np.array_equal(perm, np.arange(sim.n))          # really re-sorted
        x, v, rho, _ = sph.sph_get_state(sim.handle, sim.n, 2)
        sph.sph_build_cells(sim.handle)            # neighbour table of the moved state
        dt = 0.1 * prob.h ** 2 / 0.01
        sph.sph_diffusion_step(sim.handle, sp, dt, 5)
        Cg = sph.sph_species_get(sim.handle, sp, sim.n)
        sph.sph_species_destroy(sp)
    finally:
        sim.close()
    p = copy.copy(prob)
    p.pos, p.rho = x, rho
    p.mass = np.asarray(prob.mass, dtype=np.float32).astype(np.float64)
    Co = _oracle_run(p, 0.01 * np.eye(2), C0, dt, 5)
    assert np.max(np.abs(Cg - Co)) <= _bound(5, C0, Co)


def test_batched_tanks_diffuse_independently(sph):
    pa = _representable_problem(wk.diffusion_band(n=64, ny=64, kappa=1.0, a=0.1))
    pb = _representable_problem(wk.diffusion_band(n=48, ny=48, kappa=1.0, a=0.2))
    D = np.eye(2)
    dt = 0.1 * min(pa.h, pb.h) ** 2          # the smaller of the two stable steps
    C0 = np.concatenate([pa.meta["C0"], pb.meta["C0"]])
    Cg = _gpu_run(sph, [pa, pb], D, C0, dt, 8)
    Ca = _oracle_run(pa, D, pa.meta["C0"], dt, 8)
    Cb = _oracle_run(pb, D, pb.meta["C0"], dt, 8)
    Co = np.concatenate([Ca, Cb])
    assert np.max(np.abs(Cg - Co)) <= _bound(8, C0, Co)


def test_edge_cases(sph):
    # zero steps leave C as set; a lone particle has no neighbours; bad arguments fail cleanly
    prob = _representable_problem(wk.diffusion_band(n=32, ny=32))
    sim = sph.Simulation(prob)
    try:
        sp = sph.sph_species_create(sim.handle, np.eye(2), 2)
        C0 = prob.meta["C0"]
        sph.sph_species_set(sim.handle, sp, C0)
        with pytest.raises(sph.SphError):                     # no neighbour table yet
            sph.sph_diffusion_step(sim.handle, sp, 1e-5, 1)
        sph.sph_build_cells(sim.handle)
        sph.sph_diffusion_step(sim.handle, sp, 1e-5, 0)
        assert np.array_equal(sph.sph_species_get(sim.handle, sp, sim.n), C0)
        for dt in (0.0, -1.0, float("nan")):
            with pytest.raises(sph.SphError):
                sph.sph_diffusion_step(sim.handle, sp, dt, 1)
        sph.sph_species_destroy(sp)
        for bad in ([[1.0, 2.0], [2.0, 1.0]], [[1.0, 0.1], [0.0, 1.0]]):
            with pytest.raises(sph.SphError):
                sph.sph_species_create(sim.handle, np.asarray(bad), 2)
    finally:
        sim.close()
    one = copy.copy(prob)
    one.pos, one.vel, one.rho, one.mass = prob.pos[:1], prob.vel[:1], prob.rho[:1], prob.mass[:1]
    Cg = _gpu_run(sph, one, np.eye(2), np.array([0.75]), 1e-5, 4)
    assert Cg[0] == 0.75


def _patch_oracle_one_step(x, C0, m, rho, D, dt, prm_full, centres):
    """One RK2 step evaluated exactly at each centre from the particles within 4h of it
    (two hops of the 2h support), on the unwrapped periodic neighbourhood."""
    from scipy.spatial import cKDTree
    tree = cKDTree(np.mod(x, 1.0), boxsize=1.0)
    R = 4.0 * prm_full.h * (1.0 + 1e-6) + 2 * prm_full.dp
    out = []
    for c in centres:
        idx = np.asarray(tree.query_ball_point(np.mod(x[c], 1.0), R), dtype=np.int64)
        rel = x[idx] - x[c]
        rel -= np.round(rel)
        d = x.shape[1]
        prm = o.Params(dim=d, h=prm_full.h, dp=prm_full.dp, rho0=prm_full.rho0, c0=prm_full.c0,
                       cfl_ad=0.25, cfl_ac=0.6, u_ref=1.0, nu=0.0, gravity=np.zeros(d),
                       lo=np.full(d, -1.0), hi=np.full(d, 1.0), periodic=np.zeros(d, bool),
                       free_surface=False)
        I, J = df.fluid_pairs(rel, prm)
        vol = m[idx] / rho[idx]
        C1 = df.rk2_step(rel, C0[idx], vol, I, J, df.tensor_inverse(D, d), dt, prm)
        out.append(C1[int(np.nonzero(idx == c)[0][0])])
    return np.asarray(out)


def test_full_size_block_sampled_and_analytic(sph):
    # the 3D diffusion workload at full size (200^3 = 8.0M particles): one step against the
    # oracle on 48 sampled particles, then the Gaussian blob against its closed form
    prob = wk.diffusion_block_3d(200, kappa=1.0, sigma=0.1)
    p = _representable_problem(prob)
    C0 = np.asarray(prob.meta["C0"], dtype=np.float32).astype(np.float64)
    D = np.eye(3)
    dt = prob.meta["dt"]
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, D, 3)
        sph.sph_species_set(sim.handle, sp, C0)
        sph.sph_diffusion_step(sim.handle, sp, dt, 1)
        C1 = sph.sph_species_get(sim.handle, sp, sim.n)
        sph.sph_diffusion_step(sim.handle, sp, dt, 19)
        C20 = sph.sph_species_get(sim.handle, sp, sim.n)
        sph.sph_species_destroy(sp)
    finally:
        sim.close()
    rng = np.random.default_rng(11)
    centre = np.argmin(np.sum((p.pos - 0.5) ** 2, axis=1))
    sample = np.concatenate([[centre], rng.choice(sim.n, 47, replace=False)])
    prm = o.Params.from_problem(p)
    want = _patch_oracle_one_step(p.pos, C0, p.mass, p.rho, D, dt, prm, sample)
    got = C1[sample]
    assert np.max(np.abs(got - want)) <= 8 * 2.0 ** -24 + 1e-5 * np.max(np.abs(want - C0[sample]))
    # Gaussian blob: C = (s0^2/s^2)^(3/2) exp(-r^2 / (2 s^2)), s^2 = s0^2 + 2 kappa t; the
    # lattice at h = 1.3 dp diffuses about 2 % slower (about 5e-4 here); a factor-2 slip
    # in the operator would show as about 2.5e-2
    t = 20 * dt
    s2 = 0.01 + 2.0 * t
    r2 = np.sum((p.pos - 0.5) ** 2, axis=1)
    exact = (0.01 / s2) ** 1.5 * np.exp(-r2 / (2 * s2))
    assert np.max(np.abs(C20 - exact)) < 2e-3
    assert abs(np.sum(C20) / np.sum(C0) - 1.0) < 1e-5      # uniform volumes: sum C conserved


@pytest.mark.parametrize("name", ["aniso2d", "iso3d", "band2d"])
def test_per_particle_diffusivity_matches_oracle(sph, name):
    # reading R17: per-particle factors s_i on the tensor; the band has uniform volumes, so
    # only the factors take it off the uniform path
    p, D, C0, dt = _case(name)
    s = np.random.default_rng(13).uniform(0.5, 2.0, p.n_fluid).astype(np.float32).astype(np.float64)
    dt = dt / 2.0                                   # s up to 2
    steps = 10
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, D, sim.dim)
        try:
            sph.sph_species_set(sim.handle, sp, C0)
            sph.sph_species_set_scale(sim.handle, sp, s)
            sph.sph_diffusion_step(sim.handle, sp, dt, steps)
            Cg = sph.sph_species_get(sim.handle, sp, sim.n)
            with pytest.raises(sph.SphError):          # a non-positive factor is rejected
                sph.sph_species_set_scale(sim.handle, sp, np.where(np.arange(sim.n) == 7, 0.0, 1.0))
        finally:
            sph.sph_species_destroy(sp)
    finally:
        sim.close()
    prm = o.Params.from_problem(p)
    Co = df.run(p.pos, C0, p.mass, p.rho, np.asarray(D)[:p.dim, :p.dim], dt, steps, prm, scale=s)
    assert np.max(np.abs(Co - C0)) > 1e-3
    assert np.max(np.abs(Cg - Co)) <= _bound(steps, C0, Co), (name, np.max(np.abs(Cg - Co)))


@pytest.mark.parametrize("name", ["patch2d", "band2d", "aniso2d", "iso3d", "aniso3d"])
def test_corrected_diffusion_matches_oracle(sph, name):
    # Eq. grad-laplace-renormalize under reading R31; on the free-edged patch B0 varies near
    # the edges (and the masses are jittered), on the periodic bodies it does not
    if name == "patch2d":
        p = _representable_problem(wk.diffusion_patch(48), mass_jitter=0.1, seed=2)
        C0 = np.asarray(np.random.default_rng(11).uniform(0.0, 1.0, p.n_fluid), np.float32).astype(np.float64)
        D = np.eye(2)
        dt = 0.1 * p.h ** 2
    else:
        p, D, C0, dt = _case(name)
    steps = 10
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, D, sim.dim)
        try:
            sph.sph_species_set_correction(sim.handle, sp, True)
            sph.sph_species_set(sim.handle, sp, C0)
            sph.sph_diffusion_step(sim.handle, sp, dt, steps)
            Cg = sph.sph_species_get(sim.handle, sp, sim.n)
            sph.sph_species_set(sim.handle, sp, np.full(sim.n, 0.75))   # a constant stays put
            sph.sph_diffusion_step(sim.handle, sp, dt, 3)
            assert np.array_equal(sph.sph_species_get(sim.handle, sp, sim.n), np.full(sim.n, 0.75))
        finally:
            sph.sph_species_destroy(sp)
    finally:
        sim.close()
    prm = o.Params.from_problem(p)
    Co = df.run(p.pos, C0, p.mass, p.rho, np.asarray(D)[:p.dim, :p.dim], dt, steps, prm, corrected=True)
    Cp = df.run(p.pos, C0, p.mass, p.rho, np.asarray(D)[:p.dim, :p.dim], dt, steps, prm)
    err = np.max(np.abs(Cg - Co))
    print(f"{name}: corrected vs oracle {err:.2e} (bound {_bound(steps, C0, Co):.2e}); "
          f"corrected - plain {np.max(np.abs(Co - Cp)):.2e}")
    assert np.max(np.abs(Co - C0)) > 1e-3
    assert np.max(np.abs(Co - Cp)) > 10 * _bound(steps, C0, Co)      # the correction shows
    assert err <= _bound(steps, C0, Co), (name, err)


@pytest.mark.parametrize("name,scale,corrected", [("aniso2d", False, False), ("iso3d", False, False),
                                                  ("aniso2d", True, False), ("patch2d", False, True),
                                                  ("aniso3d", True, True)])
def test_per_particle_tensors_match_oracle(sph, name, scale, corrected):
    # reading R32: every particle its own SPD tensor, alone, with diffusivity factors on top
    # (D_i = s_i Dp_i) and with the kernel-corrected form
    if name == "patch2d":
        p = _representable_problem(wk.diffusion_patch(48), mass_jitter=0.1, seed=2)
        C0 = np.asarray(np.random.default_rng(11).uniform(0.0, 1.0, p.n_fluid), np.float32).astype(np.float64)
    else:
        p, _, C0, _ = _case(name)
    rng = np.random.default_rng(21)
    d = p.dim
    A = rng.normal(size=(p.n_fluid, d, d))
    Dp = 0.3 * (A @ np.swapaxes(A, 1, 2)) + 0.5 * np.eye(d)
    Dp = 0.5 * (Dp + np.swapaxes(Dp, 1, 2))
    s = rng.uniform(0.5, 2.0, p.n_fluid).astype(np.float32).astype(np.float64) if scale else None
    lam = max(float(np.max(np.linalg.eigvalsh(Dp))) * (2.0 if scale else 1.0), 1e-12)
    dt = 0.1 * p.h ** 2 / lam
    steps = 10
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, np.eye(d), sim.dim)
        try:
            sph.sph_species_set_tensors(sim.handle, sp, Dp)
            if s is not None:
                sph.sph_species_set_scale(sim.handle, sp, s)
            if corrected:
                sph.sph_species_set_correction(sim.handle, sp, True)
            bad = Dp.copy()
            bad[3] = -np.eye(d)
            with pytest.raises(sph.SphError):          # not positive definite: refused, tensors kept
                sph.sph_species_set_tensors(sim.handle, sp, bad)
            sph.sph_species_set(sim.handle, sp, C0)
            sph.sph_diffusion_step(sim.handle, sp, dt, steps)
            Cg = sph.sph_species_get(sim.handle, sp, sim.n)
        finally:
            sph.sph_species_destroy(sp)
    finally:
        sim.close()
    prm = o.Params.from_problem(p)
    Co = df.run(p.pos, C0, p.mass, p.rho, np.eye(d), dt, steps, prm, scale=s, corrected=corrected, tensors=Dp)
    err = np.max(np.abs(Cg - Co))
    print(f"{name} scale {scale} corrected {corrected}: tensors vs oracle {err:.2e} (bound {_bound(steps, C0, Co):.2e})")
    assert np.max(np.abs(Co - C0)) > 1e-3
    assert err <= _bound(steps, C0, Co), (name, err)


def test_clearing_tensors_returns_to_the_species_tensor(sph):
    p, D, C0, dt = _case("aniso2d")
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        out = []
        for with_tensors in (False, True):
            sp = sph.sph_species_create(sim.handle, D, sim.dim)
            try:
                if with_tensors:
                    sph.sph_species_set_tensors(sim.handle, sp, np.broadcast_to(2.0 * np.eye(2), (p.n_fluid, 2, 2)))
                    sph.sph_species_set_tensors(sim.handle, sp, None)
                sph.sph_species_set(sim.handle, sp, C0)
                sph.sph_diffusion_step(sim.handle, sp, dt, 5)
                out.append(sph.sph_species_get(sim.handle, sp, sim.n))
            finally:
                sph.sph_species_destroy(sp)
    finally:
        sim.close()
    assert np.array_equal(out[0], out[1])


def test_uniform_factor_equals_scaled_tensor(sph):
    # a factor equal for every particle matches the tensor scaled by it
    p, D, C0, dt = _case("iso3d")
    a = _gpu_run(sph, p, 2.0 * np.asarray(D), C0, dt / 2, 6)
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, D, 3)
        sph.sph_species_set(sim.handle, sp, C0)
        sph.sph_species_set_scale(sim.handle, sp, np.full(sim.n, 2.0))
        sph.sph_diffusion_step(sim.handle, sp, dt / 2, 6)
        b = sph.sph_species_get(sim.handle, sp, sim.n)
        sph.sph_species_destroy(sp)
    finally:
        sim.close()
    assert np.max(np.abs(a - b)) <= 8 * 6 * 2.0 ** -24 * np.max(np.abs(C0))


def test_failed_factor_upload_leaves_no_factors(sph):
    # header contract: a set_scale call that fails returns SPH_E_INVALID and leaves no factors,
    # both on the first call (nothing allocated before) and after factors were set
    p, D, C0, dt = _case("iso3d")
    ref = _gpu_run(sph, p, D, C0, dt, 4)
    sim = sph.Simulation(p)
    try:
        sph.sph_build_cells(sim.handle)
        sp = sph.sph_species_create(sim.handle, D, 3)
        try:
            for preset in (None, np.full(sim.n, 2.0)):
                sph.sph_species_set(sim.handle, sp, C0)
                if preset is not None:
                    sph.sph_species_set_scale(sim.handle, sp, preset)
                with pytest.raises(sph.SphError) as e:
                    sph.sph_species_set_scale(sim.handle, sp, None)      # no array
                assert e.value.code == sph.SPH_E_INVALID
                sph.sph_diffusion_step(sim.handle, sp, dt, 4)
                np.testing.assert_array_equal(sph.sph_species_get(sim.handle, sp, sim.n), ref)
        finally:
            sph.sph_species_destroy(sp)
    finally:
        sim.close()
