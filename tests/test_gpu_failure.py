"""Failure detection on the GPU without a GPU fault.

The device-side substep loop has a bound (sph_params.max_substeps): an advection step that
needs more substeps ends with SPH_E_TIMEOUT and a handle that stays usable. With
SPH_FLAG_DEBUG_BOUNDS every table is checked before a kernel reads it: an out-of-range entry
planted from the host (sph_debug_write) is reported as SPH_E_BOUNDS and nothing that would
read it is launched, so no test here ever makes a kernel touch a bad address.
"""
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


@pytest.mark.parametrize("graph", [False, True])
def test_substep_bound_returns_timeout_and_the_handle_stays_valid(sph, graph):
    prob = wk.dam_break_2d(n_per_H=20)
    ref = sph.Simulation(prob)
    ref.step(1)
    assert ref.diagnostics()["substeps"] > 1          # this step needs several substeps
    ref.close()
    flags = sph.SPH_FLAG_GRAPH if graph else 0
    sim = sph.Simulation(prob, flags=flags, max_substeps=1)
    with pytest.raises(sph.SphError) as e:
        sim.step(1)
    assert e.value.code == sph.SPH_E_TIMEOUT
    sph.sph_clear_error(sim.handle)
    d = sim.diagnostics()
    assert d["substeps"] == 1 and d["advection_steps"] == 1   # stopped at the bound
    for a in sim.state():
        assert np.all(np.isfinite(a))
    with pytest.raises(sph.SphError) as e:            # the bound holds for the next step too
        sim.step(1)
    assert e.value.code == sph.SPH_E_TIMEOUT
    sph.sph_clear_error(sim.handle)
    assert sim.diagnostics()["substeps"] == 2
    sim.close()


def test_debug_bounds_catches_a_corrupted_table_before_any_kernel_reads_it(sph):
    prob = wk.dam_break_2d(n_per_H=20)
    sim = sph.Simulation(prob, flags=sph.SPH_FLAG_DEBUG_BOUNDS | sph.SPH_FLAG_GRAPH)
    sim.step(2)                                       # the library's own tables pass the checks
    plain = sph.Simulation(prob)
    plain.step(2)
    for u, v in zip(sim.state(), plain.state()):      # the checks change no result
        np.testing.assert_array_equal(u, v)
    plain.close()

    sim.build_cells()
    before = sim.state()
    fc, _, _, _ = sim.neighbours()
    assert fc.min() > 0
    # an out-of-range fluid index in slot 0 of the particle stored at position 5
    sph.sph_debug_write(sim.handle, sph.SPH_DEBUG_NEIGHBOUR, 5, 0, sim.n + 1000)
    readers = [sim.advection_step, sim.acoustic_substep, lambda: sph.sph_pair_count(sim.handle),
               lambda: sph.sph_gather_ceiling(sim.handle, 1), sim.neighbours]
    for read in readers:
        with pytest.raises(sph.SphError) as e:
            read()
        assert e.value.code == sph.SPH_E_BOUNDS
        sph.sph_clear_error(sim.handle)
    for u, v in zip(before, sim.state()):             # nothing ran on the bad table
        np.testing.assert_array_equal(u, v)
    sim.step(1)                                       # a new configuration update rebuilds it
    # a wall offset (kept from creation, read by every update) out of range: the next
    # update stops after the scan, before the neighbour search would read it
    sph.sph_debug_write(sim.handle, sph.SPH_DEBUG_WALL_OFFSET, 3, 0, 1 << 30)
    with pytest.raises(sph.SphError) as e:
        sim.build_cells()
    assert e.value.code == sph.SPH_E_BOUNDS
    sim.close()


def test_debug_write_is_refused_without_the_checks(sph):
    sim = sph.Simulation(wk.dam_break_2d(n_per_H=10))
    sim.build_cells()
    with pytest.raises(sph.SphError) as e:
        sph.sph_debug_write(sim.handle, sph.SPH_DEBUG_NEIGHBOUR, 0, 0, 0)
    assert e.value.code == sph.SPH_E_INVALID
    sim.close()
