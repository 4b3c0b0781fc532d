"""The precision argument for summing the relaxations' pair terms plainly in FP32.

The GPU's pressure relaxation adds each particle's pair terms in two FP32 lanes without
compensation. This test takes the FP64 oracle's pair terms on the parity states (and a
hydrostatic tank, where the terms cancel most), rounds them to FP32 and sums them the way
the kernel does (two interleaved lanes, sequentially, then the lanes added), and checks that
the accumulation alone stays far inside the 1e-5 per-substep tolerance."""
import copy

import numpy as np
import pytest

from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wk
from tests.parity import perturbed_state, rel_l2, walls_representable


def _case(name):
    if name == "dam2d":
        return wk.dam_break_2d(), 0.3, 0.01
    if name == "tg":
        return wk.taylor_green(64), 0.05, 0.005
    if name == "dam3d":
        return wk.dam_break_3d(16), 0.3, 0.01
    if name == "still3d":
        return wk.still_tank(dim=3, H=0.5, dp=0.025), 0.0, 0.0
    return wk.periodic_box(dim=3, n=12, seed=3), 0.1, 0.01


@pytest.mark.parametrize("name", ["dam2d", "tg", "dam3d", "box3d", "still3d"])
def test_plain_fp32_accumulation_of_the_pressure_force(name):
    prob, va, ra = _case(name)
    prob = copy.copy(prob)
    prob.wall_pos = walls_representable(prob)
    x, v, rho, drho = perturbed_state(prob, 11, va, ra)
    if name == "still3d":                       # hydrostatic: p = rho0 g (H - y)
        rho = prob.rho0 * (1.0 + prob.meta["g"] * (prob.meta["H"] - x[:, 1]) / prob.c0 ** 2)
    prm = o.Params.from_problem(prob)
    st, w = o.state_from_problem(prob)
    st.x, st.v, st.rho, st.drho = x, v, rho, drho
    I, J, _, _ = o.neighbour_sets(x, w.x, prm)
    dt = 0.5 * o.dt_acoustic(st.v, prm)
    rho_h = st.rho + 0.5 * dt * st.drho
    xh = st.x + 0.5 * dt * st.v
    p = o.eos_pressure(rho_h, prm)
    _, r, e = o._geometry(xh[I], xh[J], prm)
    dW = o.kernel_dW(r, prm.h, prm.dim)
    _, Ps = o.riemann(rho_h[I], rho_h[J], np.sum(st.v[I] * e, 1), np.sum(st.v[J] * e, 1), p[I], p[J], prm.c0)
    term = (st.m[J] / rho_h[J] * Ps)[:, None] * ((-e) * dW[:, None])      # V_j P* grad_i W_ij
    N = x.shape[0]
    exact = np.zeros((N, prm.dim))
    np.add.at(exact, I, term)
    order = np.lexsort((J, I))
    Is, Ts = I[order], term[order].astype(np.float32)
    starts = np.searchsorted(Is, np.arange(N))
    ends = np.searchsorted(Is, np.arange(N), side="right")
    lanes = [np.zeros((N, prm.dim), np.float32), np.zeros((N, prm.dim), np.float32)]
    for k in range(int((ends - starts).max())):
        idx = starts + k
        ok = idx < ends
        lanes[k % 2] += np.where(ok[:, None], Ts[np.minimum(idx, len(Ts) - 1)], np.float32(0))
    total = lanes[0].astype(np.float64) + lanes[1].astype(np.float64)
    a_exact = prm.gravity[None, :] - 2.0 / rho_h[:, None] * exact
    a_fp32 = prm.gravity[None, :] - 2.0 / rho_h[:, None] * total
    err = rel_l2(a_fp32, a_exact)
    print(f"{name}: plain FP32 accumulation, dv/dt rel L2 {err:.2e}")
    assert err < 1e-6
