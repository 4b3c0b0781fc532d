"""The allocation-free diagnostics entry point against the handle-based one.

Callers that cannot allocate device memory (inside another framework's memory
pool, under a fixed device-memory budget) use sph_diagnostics_noalloc on their
own device arrays. Its scratch is a fixed array in the library's device image
that every call reuses, so two calls in a row must both give the results of
sph_diagnostics on the same state. The file name sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2010_12375_gb300 import workloads as wk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUM_TOL = 1e-12      # both sides sum the same FP64 values, in different orders


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_12375_gb300 import sph as s
    s.load()
    return s


def _close(a, b):
    return abs(a - b) <= SUM_TOL * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("problem", ["dam2d", "dam3d"])
def test_noalloc_diagnostics_match_handle_diagnostics(sph, problem):
    prob = wk.dam_break_2d(n_per_H=20) if problem == "dam2d" else wk.dam_break_3d(12)
    params = sph.params_from(prob)
    sim = sph.Simulation(prob)
    dev = torch.device("cuda", 0)
    for call in range(2):                      # two calls in a row share the static scratch
        sim.step(4)
        ref = sim.diagnostics()
        pos, vel, rho, _ = sim.state()
        # the handle holds masses in FP32; its state's masses are those values
        mass = np.asarray(prob.mass, dtype=np.float32).astype(np.float64)
        t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (pos, vel, rho, mass)]
        got = sph.sph_diagnostics_noalloc(params, *t)
        for key in ("mass", "kinetic", "potential", "internal", "energy", "mean_rho_dev"):
            assert _close(got[key], ref[key]), (call, key, got[key], ref[key])
        for a in range(prob.dim):
            assert abs(got["momentum"][a] - ref["momentum"][a]) <= SUM_TOL * max(
                np.sum(prob.mass * np.abs(vel[:, a])), 1e-300), (call, a)
        assert got["max_rho_dev"] == ref["max_rho_dev"]
        assert got["front_x"] == ref["front_x"]
        assert got["n_fluid"] == ref["n_fluid"] == prob.n_fluid
    sim.close()


def test_noalloc_rejects_bad_arguments(sph):
    prob = wk.dam_break_2d(n_per_H=10)
    params = sph.params_from(prob)
    host = [np.ascontiguousarray(a, dtype=np.float64) for a in (prob.pos, prob.vel, prob.rho, prob.mass)]
    with pytest.raises(sph.SphError) as e:                 # host arrays would need staging
        sph.sph_diagnostics_noalloc(params, *host)
    assert e.value.code == sph.SPH_E_INVALID and "device" in str(e.value)
    params.dim = 4
    dev = [torch.from_numpy(a).cuda() for a in host]
    with pytest.raises(sph.SphError) as e:
        sph.sph_diagnostics_noalloc(params, *dev)
    assert e.value.code == sph.SPH_E_INVALID
