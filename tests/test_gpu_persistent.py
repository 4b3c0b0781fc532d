"""The persistent substep loop (SPH_FLAG_PERSISTENT): one cooperative launch per advection
step runs every tank's substeps. It runs the per-launch kernels' per-particle code, so its
results must equal the per-launch loop's bit for bit; with that, the batched tanks' parity
with the oracle (test_gpu_parity) carries over to it."""
import numpy as np
import pytest

from paper_2010_12375_gb300 import workloads as wk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _run(sph, problems, flags, steps):
    sim = sph.Simulation(problems, flags=flags)
    sim.step(steps)
    out = sim.state(), sim.diagnostics(), sim.kernel_launches()
    sim.close()
    return out


@pytest.mark.parametrize("case", ["batched16", "dam3d", "tg_transport", "single2d"])
def test_persistent_loop_equals_the_per_launch_loop(sph, case):
    if case == "batched16":
        tanks = wk.batched_dam_breaks(256)
        order = np.argsort([t.n_fluid for t in tanks], kind="stable")
        probs = [tanks[k] for k in order[np.unique(np.round(np.linspace(0, 255, 16)).astype(int))]]
        steps = 3
    elif case == "dam3d":
        probs, steps = wk.dam_break_3d(24), 3
    elif case == "tg_transport":
        probs, steps = [wk.taylor_green(48), wk.taylor_green(40)], 3
    else:
        probs, steps = wk.dam_break_2d(), 5
    a_state, a_diag, a_launch = _run(sph, probs, sph.SPH_FLAG_GRAPH, steps)
    b_state, b_diag, b_launch = _run(sph, probs, sph.SPH_FLAG_PERSISTENT, steps)
    for u, v in zip(a_state, b_state):
        np.testing.assert_array_equal(u, v)
    da = a_diag if isinstance(a_diag, list) else [a_diag]
    db = b_diag if isinstance(b_diag, list) else [b_diag]
    for x, y in zip(da, db):
        assert x["substeps"] == y["substeps"] and x["t"] == y["t"] and x["energy"] == y["energy"]
    assert b_launch < a_launch                       # one launch for all substeps of a step


def test_persistent_loop_reports_the_substep_bound(sph):
    sim = sph.Simulation(wk.dam_break_2d(n_per_H=20), flags=sph.SPH_FLAG_PERSISTENT, max_substeps=2)
    with pytest.raises(sph.SphError) as e:
        sim.step(1)
    assert e.value.code == sph.SPH_E_TIMEOUT
    sph.sph_clear_error(sim.handle)
    assert sim.diagnostics()["substeps"] == 2
    sim.close()
