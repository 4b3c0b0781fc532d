"""The C ABI without a GPU: the library builds, loads and exports every function that
include/sph.h declares, and the host-only parameter check behaves."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2010_12375_gb300 import build, sph
    if not os.path.exists(build.LIB_PATH):
        build.build()
    return sph


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("sph_create", "sph_build_cells", "sph_advection_step",
                     "sph_acoustic_substep", "sph_step", "sph_diagnostics"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert sorted(lib.EXPORTS) == declared_functions()


def test_binding_loads_without_gpu(lib):
    h = lib.load()
    assert h is not None


def test_params_check_on_host(lib):
    from paper_2010_12375_gb300 import workloads as wk
    good = lib.params_from(wk.dam_break_2d())
    assert lib.sph_params_check(good) == lib.SPH_OK
    assert lib.sph_params_check(lib.params_from(wk.taylor_green(50))) == lib.SPH_OK
    assert lib.sph_params_check(lib.params_from(wk.dam_break_3d(10))) == lib.SPH_OK
    cases = [("h", -1.0), ("h", float("nan")), ("dim", 4), ("c0", 0.0), ("cfl_ad", 0.0),
             ("cfl_ac", -0.6), ("nu", -1.0), ("capacity", -2), ("free_surface", 3),
             ("max_substeps", -1)]
    for field, val in cases:
        p = lib.params_from(wk.dam_break_2d())
        setattr(p, field, val)
        assert lib.sph_params_check(p) == lib.SPH_E_INVALID, field
    p = lib.params_from(wk.dam_break_2d())
    p.hi[0] = p.lo[0]
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID
    p = lib.params_from(wk.taylor_green(50))
    p.hi[1] = 2.0                                          # two different periods
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID
    p = lib.params_from(wk.taylor_green(50))
    p.h = 0.2                                              # fewer than 3 cells per period
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID
    p = lib.params_from(wk.dam_break_2d())
    p.u_ref = 0.0                                          # Dt_ad unbounded at rest
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID
    tg = wk.taylor_green(50)
    assert tg.p_transport > 0.0
    p = lib.params_from(tg)
    p.p_transport = -1.0                                   # background pressure below zero
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID
    p = lib.params_from(tg, flags=lib.SPH_FLAG_FROZEN_GEOMETRY)
    assert lib.sph_params_check(p) == lib.SPH_E_INVALID    # transport needs recomputed geometry
    p = lib.params_from(wk.taylor_green(50, transport=False), flags=lib.SPH_FLAG_FROZEN_GEOMETRY)
    assert lib.sph_params_check(p) == lib.SPH_OK


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2010_12375_gb300 import workloads as wk
    with pytest.raises(lib.SphError) as e:
        lib.Simulation(wk.dam_break_2d(n_per_H=5))
    assert e.value.code in (lib.SPH_E_CUDA, lib.SPH_E_OOM)


def test_species_and_reaction_entry_points_reject_null_handles(lib):
    # argument checks run before any CUDA call, so they are testable without a GPU
    import ctypes
    L = lib.load()
    out = ctypes.c_void_p(123)
    D = (ctypes.c_double * 4)(1.0, 0.0, 0.0, 1.0)
    assert L.sph_species_create(None, D, ctypes.byref(out)) == lib.SPH_E_INVALID
    assert out.value is None                                  # cleared on failure
    assert L.sph_species_create(None, D, None) == lib.SPH_E_INVALID
    r = lib.reaction_from(lib.SPH_REACTION_FN, a=0.1)
    assert L.sph_reaction_step(None, None, ctypes.byref(r), 0.1, 1, None) == lib.SPH_E_INVALID
    assert L.sph_diffusion_step(None, None, 0.1, 1, None) == lib.SPH_E_INVALID
    assert L.sph_species_set_correction(None, None, 1) == lib.SPH_E_INVALID
    assert L.sph_species_set_tensors(None, None, None, None) == lib.SPH_E_INVALID
    buf = (ctypes.c_double * 4)()
    for fn in (L.sph_species_set, L.sph_species_get, L.sph_species_set_gate, L.sph_species_get_gate):
        assert fn(None, None, buf, None) == lib.SPH_E_INVALID
    L.sph_species_destroy(None)                               # a no-op
    assert L.sph_species_last_error(None) == b"null species"


def test_error_control_entry_points_reject_null_handles(lib):
    L = lib.load()
    assert L.sph_clear_error(None, None) == lib.SPH_E_INVALID
    g = (ctypes.c_double * 3)(0.0, -1.0, 0.0)
    assert L.sph_set_gravity(None, -1, g, None) == lib.SPH_E_INVALID
    assert L.sph_debug_write(None, lib.SPH_DEBUG_NEIGHBOUR, 0, 0, 0, None) == lib.SPH_E_INVALID
    p = lib.params_from(__import__("paper_2010_12375_gb300.workloads", fromlist=["x"]).dam_break_2d(),
                        max_substeps=1)
    assert p.max_substeps == 1 and lib.sph_params_check(p) == lib.SPH_OK


def test_solid_entry_points_reject_null_handles(lib):
    L = lib.load()
    assert L.sph_solid_size(None) == -1
    out = ctypes.c_void_p(0)
    assert L.sph_solid_create(None, None, 0, None, None, None, None, ctypes.byref(out)) == lib.SPH_E_INVALID
    assert L.sph_solid_get_state(None, None, None, None, None, None, None, None) == lib.SPH_E_INVALID
    L.sph_solid_destroy(None)                                 # a no-op


def test_binding_rejects_caller_arrays_of_the_wrong_size(lib):
    # the C side reads or writes exactly the counts a handle implies and cannot check them:
    # the binding refuses any other size, dtype or layout before the call
    import numpy as np
    torch = pytest.importorskip("torch")
    assert lib._sized(None, 5, "x") is None
    assert lib._sized(np.zeros((2, 3)), 6, "x").shape == (2, 3)
    assert lib._sized(torch.zeros(6), 6, "x").numel() == 6
    for bad in (np.zeros(5), np.zeros(7), torch.zeros(2, 2)):
        with pytest.raises(lib.SphError) as e:
            lib._sized(bad, 6, "pos")
        assert e.value.code == lib.SPH_E_INVALID
    assert lib._out(np.zeros(4), 4, "rho").size == 4
    assert lib._out(torch.zeros(4, dtype=torch.float64), 4, "rho").numel() == 4
    for bad in (np.zeros(4, dtype=np.float32), np.zeros((4, 2))[:, 0], torch.zeros(4), np.zeros(3)):
        with pytest.raises(lib.SphError) as e:
            lib._out(bad, 4, "rho")
        assert e.value.code == lib.SPH_E_INVALID
    # the learned network's weight vector has a fixed length
    with pytest.raises(lib.SphError) as e:
        lib.sph_learned_create(2, np.zeros(lib.sph_learned_weight_count() - 1))
    assert e.value.code == lib.SPH_E_INVALID
