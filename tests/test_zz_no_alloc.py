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


def test_noalloc_large_count_uses_the_capped_grid_and_allocates_nothing(sph):
    # 3M particles: more than the 1024 blocks x 2048 particles the fixed scratch rows cover in
    # one pass, so the grid-stride loop does the rest. Reference: float64 torch sums of the same
    # formulas. Around a call (after the first, which looks the scratch address up) the device's
    # free memory does not change.
    n = 3_000_000
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(2010)
    pos = torch.rand((n, 3), dtype=torch.float64, device=dev, generator=g) * 2.0
    vel = torch.rand((n, 3), dtype=torch.float64, device=dev, generator=g) - 0.5
    rho = 1.0 + 0.04 * (torch.rand(n, dtype=torch.float64, device=dev, generator=g) - 0.5)
    mass = 1e-6 * (1.0 + torch.rand(n, dtype=torch.float64, device=dev, generator=g))
    prob = wk.dam_break_3d(12)
    params = sph.params_from(prob)
    rho0, c0 = float(prob.rho0), float(prob.c0)
    grav = torch.tensor(list(prob.gravity)[:3], dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    sph.sph_diagnostics_noalloc(params, pos, vel, rho, mass)     # first call on the device
    unchanged = False
    for _ in range(3):         # another process on the same GPU could move the figure once
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        got = sph.sph_diagnostics_noalloc(params, pos, vel, rho, mass)
        free1 = torch.cuda.mem_get_info(dev)[0]
        if free0 == free1:
            unchanged = True
            break
    assert unchanged, "free device memory changed across the call"
    dev_ = rho / rho0 - 1.0
    ref = {
        "mass": mass.sum().item(),
        "kinetic": (0.5 * mass * (vel * vel).sum(dim=1)).sum().item(),
        "potential": (-(mass * (pos @ grav))).sum().item(),
        "internal": (mass * c0 * c0 * (torch.log1p(dev_) - dev_ / (1.0 + dev_))).sum().item(),
        "mean_rho_dev": dev_.abs().mean().item(),
    }
    for key, val in ref.items():
        assert _close(got[key], val), (key, got[key], val)
    mom = (mass[:, None] * vel).sum(dim=0).cpu().numpy()
    scale = (mass[:, None] * vel.abs()).sum(dim=0).cpu().numpy()
    assert np.all(np.abs(np.asarray(got["momentum"]) - mom) <= SUM_TOL * scale)
    assert got["max_rho_dev"] == dev_.abs().max().item()
    assert got["front_x"] == pos[:, 0].max().item()
    assert got["n_fluid"] == n


def test_noalloc_rejects_bad_arguments(sph):
    import ctypes
    prob = wk.dam_break_2d(n_per_H=10)
    params = sph.params_from(prob)
    host = [np.ascontiguousarray(a, dtype=np.float64) for a in (prob.pos, prob.vel, prob.rho, prob.mass)]
    n = host[2].shape[0]
    lib = sph.load()
    out = sph.SphDiag()
    # the C entry point itself refuses host memory (it would have to stage it)
    code = lib.sph_diagnostics_noalloc(ctypes.byref(params), n, *[a.ctypes.data for a in host],
                                       ctypes.byref(out), None)
    assert code == sph.SPH_E_INVALID and "device" in lib.sph_last_error(None).decode()
    dev = [torch.from_numpy(a).cuda() for a in host]
    # the binding checks what the C call cannot see: type, layout and sizes of every array
    bad_cases = [
        [dev[0].float(), dev[1], dev[2], dev[3]],                 # float32 positions
        [dev[0], dev[1], dev[2], dev[3][:-1]],                    # one mass short
        [dev[0][:-1], dev[1], dev[2], dev[3]],                    # one position row short
        [dev[0].t(), dev[1], dev[2], dev[3]],                     # not contiguous
        [host[0], dev[1], dev[2], dev[3]],                        # a host array
    ]
    for args in bad_cases:
        with pytest.raises(sph.SphError) as e:
            sph.sph_diagnostics_noalloc(params, *args)
        assert e.value.code == sph.SPH_E_INVALID
    params.dim = 4
    with pytest.raises(sph.SphError) as e:
        sph.sph_diagnostics_noalloc(params, *dev)
    assert e.value.code == sph.SPH_E_INVALID
