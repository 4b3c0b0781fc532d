"""GPU parity of the particle gradients (Eqs. gradsph-strong, gradsph-weak; reading R18)
through sph_gradient_diagnostics, against the FP64 oracle on the same representable state.

Tolerance: 1e-5 relative L2 per field, as for the substep quantities. Each field is a sum of
20-80 pair terms with a few FP32 roundings each, Kahan-compensated; the weak density
gradient adds 2 rho0 S, S = sum V_j grad W, whose terms cancel (to the lattice's irregularity),
so its absolute error is of order eps 2 rho0 sum |V_j grad W|, about 1e-6 of the field where
the jittered lattice makes S visible and far below it elsewhere.
"""
import copy

import numpy as np
import pytest

from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import REL_L2_TOL, perturbed_state, rel_l2, representable, walls_representable

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("rho_strong", "rho_weak", "p_strong", "p_weak")


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _prepared(prob, seed):
    prob = copy.copy(prob)
    prob.wall_pos = walls_representable(prob)
    x, v, rho, _ = perturbed_state(prob, seed, 0.1, 0.02)
    x = x + np.random.default_rng(seed + 1).uniform(-0.1, 0.1, size=x.shape) * prob.dp
    if np.any(prob.periodic[:prob.dim]):
        x = np.mod(x, 1.0)
    xq, v32, rho32, _ = representable(prob, x, v, rho)
    return prob, xq, v32, rho32


def _oracle(prob, xq, rho32):
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    st.x, st.rho = xq, rho32
    st.m = np.asarray(prob.mass, dtype=np.float32).astype(np.float64)
    return o.gradients(st, w, o.neighbour_sets_quantised(st.x, w.x, prm), prm)


@pytest.mark.parametrize("case", ["dam2d", "dam3d", "tg"])
def test_gradients_match_the_oracle(sph, case):
    prob = {"dam2d": lambda: wk.dam_break_2d(),
            "dam3d": lambda: wk.dam_break_3d(16),
            "tg": lambda: wk.taylor_green(64)}[case]()
    prob, xq, v32, rho32 = _prepared(prob, 41)
    sim = sph.Simulation(prob)
    sim.set_state(xq, v32, rho32, None, t=0.0)
    sim.build_cells()
    got = sph.sph_gradient_diagnostics(sim.handle, sim.n, sim.dim)
    sim.close()
    ref = _oracle(prob, xq, rho32)
    errs = {k: rel_l2(got[k], ref[k]) for k in FIELDS}
    print(case, {k: f"{v:.2e}" for k, v in errs.items()})
    for k in FIELDS:
        assert errs[k] < REL_L2_TOL, (k, errs[k])


def test_gradients_of_batched_tanks_match_the_oracle_per_tank(sph):
    tanks = [_prepared(t, 50 + k) for k, t in enumerate(wk.batched_dam_breaks(3, n_min=800, n_max=4000))]
    sim = sph.Simulation([t[0] for t in tanks])
    sim.set_state(np.concatenate([t[1] for t in tanks]), np.concatenate([t[2] for t in tanks]),
                  np.concatenate([t[3] for t in tanks]), None, t=0.0)
    sim.build_cells()
    got = sph.sph_gradient_diagnostics(sim.handle, sim.n, sim.dim)
    off = sim.fluid_offsets
    sim.close()
    for k, (prob, xq, _, rho32) in enumerate(tanks):
        ref = _oracle(prob, xq, rho32)
        for f in FIELDS:
            assert rel_l2(got[f][off[k]:off[k + 1]], ref[f]) < REL_L2_TOL, (k, f)


def test_gradients_need_a_table_and_refuse_foreign_outputs(sph):
    sim = sph.Simulation(wk.dam_break_2d(n_per_H=10))
    with pytest.raises(sph.SphError) as e:           # no configuration update yet
        sph.sph_gradient_diagnostics(sim.handle, sim.n, sim.dim)
    assert e.value.code == sph.SPH_E_INVALID
    sim.build_cells()
    a = sph.sph_gradient_diagnostics(sim.handle, sim.n, sim.dim)
    # device outputs give the same values as host outputs
    dev = {k: torch.empty((sim.n, sim.dim), dtype=torch.float64, device="cuda") for k in FIELDS}
    lib = sph.load()
    assert lib.sph_gradient_diagnostics(sim.handle, *[dev[k].data_ptr() for k in FIELDS], None) == sph.SPH_OK
    for k in FIELDS:
        np.testing.assert_array_equal(dev[k].cpu().numpy(), a[k])
    sim.close()
