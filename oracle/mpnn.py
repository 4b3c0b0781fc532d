"""FP64 CPU oracle of the learned stand-in for the acoustic substeps (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU leg may use this module.

A message-passing network over the frozen SPH neighbour graph of an advection step
predicts each fluid particle's change of velocity and density over the whole step.
The paper has no learned component; this network is the project's own definition,
and this module is its plain reference (forward and hand-written backward), pinned
against central finite differences.

Definition (d = dimension, F = 64 hidden width, R = 3 rounds with shared weights;
every layer's input carries a trailing 1 so its bias is the last weight column; inputs
are zero-padded to the matrix widths K below):
  node input   u_i = [v_i/c0, S_RHO (rho_i/rho0 - 1), dt_ad c0/h, 1]            (K = 16)
  edge input   x_ij = [r_ij/h, (v_i - v_j)/c0, S_RHO dev_i, S_RHO dev_j, wall]   (2d + 3)
               walls: v_j = 0, dev_j = 0, wall = 1; r_ij = r_i - r_j
  encoder      h_i = relu(W_enc u_i)
  round        z_ij = relu(W_e1 [x_ij, h_j, 1])       (h_j = 0 for walls; K = 80)
               m_ij = W_e2 [z_ij, 1]                   (K = 80)
               a_i  = (1 / NBAR) sum_j m_ij            (fluid and wall neighbours)
               h_i += W_n2 [relu(W_n1 [h_i, a_i, 1]), 1]   (K = 144, 80)
  decoder      y_i = W_d2 [relu(W_d1 [h_i, 1]), 1]     (K = 80, 80; the first d + 1 of its
                                                       16 output rows are used)
  targets      y_i = [(dv_i - g dt_ad) / V_S, S_RHO drho_i / rho0], V_S = |g| dt_ad
               (U_ref when g = 0): the velocity change is measured in units of gravity's
  loss         mean over particles and outputs of (y_i - target_i)^2
Every matrix product rounds both operands to bfloat16 (round to nearest even) and
accumulates exactly; backward treats the rounding as the identity. With `bf16=False`
the network is plain FP64 (used for the finite-difference pin). Weights are stored in the
order enc, e1, e2, n1, n2, d1, d2, each row-major (outputs x padded inputs): 32,000 floats.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

F = 64
ROUNDS = 3
S_RHO = 100.0
K_ENC, K_E1, K_E2, K_N1, K_N2, K_D1, K_D2 = 16, 80, 80, 144, 80, 80, 80


def nbar(dim: int) -> float:
    """Aggregation normaliser: the interior neighbour count at h = 1.3 dp."""
    return 20.0 if dim == 2 else 80.0


def layer_shapes(dim: int):
    """(rows = outputs, cols = padded inputs) of every weight matrix, in storage order."""
    return {"enc": (F, K_ENC), "e1": (F, K_E1), "e2": (F, K_E2), "n1": (F, K_N1),
            "n2": (F, K_N2), "d1": (F, K_D1), "d2": (16, K_D2)}


def init_weights(dim: int, seed: int = 0):
    """He-style initialisation of the live input columns; padding columns are zero."""
    rng = np.random.default_rng(seed)
    live = {"enc": dim + 3, "e1": 2 * dim + 3 + F + 1, "e2": F + 1, "n1": 2 * F + 1,
            "n2": F + 1, "d1": F + 1, "d2": F + 1}
    W = {}
    for name, (r, c) in layer_shapes(dim).items():
        w = np.zeros((r, c))
        fan = live[name]
        w[:, :fan] = rng.normal(0.0, np.sqrt(2.0 / fan), size=(r, fan))
        w[:, fan - 1] = 0.0                                    # biases start at zero
        if name in ("e2", "n2", "d2"):
            w *= 0.1                                           # small residual / output layers
        if name == "d2":
            w[dim + 1:, :] = 0.0                               # unused output rows
        W[name] = w
    return W


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest even) and return as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@dataclass
class Graph:
    """The inputs of one sample: node and edge features and the edge list (edges of a
    node are contiguous, in the node's neighbour order)."""
    dim: int
    u: np.ndarray            # (N, K_ENC) node inputs (padded, trailing 1 at column dim + 2)
    x: np.ndarray            # (E, 2d+3) edge features
    src: np.ndarray          # (E,) node i of each edge
    nbr: np.ndarray          # (E,) fluid neighbour j, or -1 for a wall
    n: int


def build_graph(dim, pos, vel, rho, wall_pos, I, J, IW, KW, h, c0, rho0, dt_ad):
    """Features of the sample whose fluid pairs are (I, J) and wall pairs (IW, KW), edges
    ordered by node, then fluid neighbours before walls (each group in the given order)."""
    n = pos.shape[0]
    dev = rho / rho0 - 1.0
    u = np.zeros((n, K_ENC))
    u[:, :dim] = vel / c0
    u[:, dim] = S_RHO * dev
    u[:, dim + 1] = dt_ad * c0 / h
    u[:, dim + 2] = 1.0
    rows = []
    for group, (a, b) in enumerate(((I, J), (IW, KW))):
        order = np.lexsort((np.arange(a.size), a))          # by node, stable
        a, b = a[order], b[order]
        xe = np.zeros((a.size, 2 * dim + 3))
        if group == 0:
            xe[:, :dim] = (pos[a] - pos[b]) / h
            xe[:, dim:2 * dim] = (vel[a] - vel[b]) / c0
            xe[:, 2 * dim + 1] = S_RHO * dev[b]
            nb = b.astype(np.int64)
        else:
            xe[:, :dim] = (pos[a] - wall_pos[b]) / h
            xe[:, dim:2 * dim] = vel[a] / c0
            xe[:, 2 * dim + 2] = 1.0
            nb = np.full(a.size, -1, dtype=np.int64)
        xe[:, 2 * dim] = S_RHO * dev[a]
        rows.append((a, xe, nb))
    src = np.concatenate([rows[0][0], rows[1][0]])
    x = np.concatenate([rows[0][1], rows[1][1]])
    nb = np.concatenate([rows[0][2], rows[1][2]])
    order = np.argsort(src, kind="stable")                  # node-major, fluid before wall
    return Graph(dim=dim, u=u, x=x[order], src=src[order], nbr=nb[order], n=n)


def _mm(X, W, q):
    """X @ W.T with both operands rounded to bfloat16 when q, exact accumulation."""
    if q:
        return bf16(X) @ bf16(W).T
    return X @ W.T


def forward(W, g: Graph, q: bool = True):
    """Returns the outputs (N, d+1) and the activations the backward pass needs."""
    dim, n, E = g.dim, g.n, g.src.size
    nb = nbar(dim)
    cache = {"h": [], "XE": [], "Z1": [], "XN": [], "Z2": []}
    z0 = _mm(g.u, W["enc"], q)
    h = np.maximum(z0, 0.0)
    cache["z0"] = z0
    fe = 2 * dim + 3
    for _ in range(ROUNDS):
        XE = np.zeros((E, K_E1))
        XE[:, :fe] = g.x
        fl = g.nbr >= 0
        XE[fl, fe:fe + F] = h[g.nbr[fl]]
        XE[:, fe + F] = 1.0
        Z1 = _mm(XE, W["e1"], q)
        A1 = np.zeros((E, K_E2))
        A1[:, :F] = np.maximum(Z1, 0.0)
        A1[:, F] = 1.0
        M = _mm(A1, W["e2"], q)
        a = np.zeros((n, F))
        np.add.at(a, g.src, M)
        a /= nb
        XN = np.zeros((n, K_N1))
        XN[:, :F] = h
        XN[:, F:2 * F] = a
        XN[:, 2 * F] = 1.0
        Z2 = _mm(XN, W["n1"], q)
        A2 = np.zeros((n, K_N2))
        A2[:, :F] = np.maximum(Z2, 0.0)
        A2[:, F] = 1.0
        cache["h"].append(h)
        cache["XE"].append(XE)
        cache["Z1"].append(Z1)
        cache["XN"].append(XN)
        cache["Z2"].append(Z2)
        h = h + _mm(A2, W["n2"], q)
    XD = np.zeros((n, K_D1))
    XD[:, :F] = h
    XD[:, F] = 1.0
    Z3 = _mm(XD, W["d1"], q)
    A3 = np.zeros((n, K_D2))
    A3[:, :F] = np.maximum(Z3, 0.0)
    A3[:, F] = 1.0
    Y = _mm(A3, W["d2"], q)[:, :dim + 1]
    cache.update(h_final=h, XD=XD, Z3=Z3, A3=A3)
    return Y, cache


def loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def backward(W, g: Graph, cache, Y, T, q: bool = True):
    """Gradients of the loss with respect to every weight matrix. Each product rounds both
    of its operands to bfloat16 (the upstream gradient included) and the rounding is the
    identity for differentiation (straight-through)."""
    dim, n = g.dim, g.n
    nb = nbar(dim)
    Wq = {k: (bf16(v) if q else v) for k, v in W.items()}
    rnd = (lambda a: bf16(a)) if q else (lambda a: a)
    dW = {k: np.zeros_like(v) for k, v in W.items()}
    dY = np.zeros((n, 16))
    dY[:, :dim + 1] = 2.0 * (Y - T) / Y.size
    dW["d2"] += rnd(dY).T @ rnd(cache["A3"])
    dA3 = rnd(dY) @ Wq["d2"]
    dZ3 = dA3[:, :F] * (cache["Z3"] > 0)
    dW["d1"] += rnd(dZ3).T @ rnd(cache["XD"])
    dh = (rnd(dZ3) @ Wq["d1"])[:, :F]
    fe = 2 * dim + 3
    for r in reversed(range(ROUNDS)):
        h, XE, Z1, XN, Z2 = (cache["h"][r], cache["XE"][r], cache["Z1"][r], cache["XN"][r],
                             cache["Z2"][r])
        # h_new = h + W_n2 [relu(Z2), 1]
        A2 = np.zeros((n, K_N2))
        A2[:, :F] = np.maximum(Z2, 0.0)
        A2[:, F] = 1.0
        dW["n2"] += rnd(dh).T @ rnd(A2)
        dA2 = rnd(dh) @ Wq["n2"]
        dZ2 = dA2[:, :F] * (Z2 > 0)
        dW["n1"] += rnd(dZ2).T @ rnd(XN)
        dXN = rnd(dZ2) @ Wq["n1"]
        dh_prev = dh + dXN[:, :F]
        da = dXN[:, F:2 * F] / nb
        dM = da[g.src]
        A1 = np.zeros((XE.shape[0], K_E2))
        A1[:, :F] = np.maximum(Z1, 0.0)
        A1[:, F] = 1.0
        dW["e2"] += rnd(dM).T @ rnd(A1)
        dA1 = rnd(dM) @ Wq["e2"]
        dZ1 = dA1[:, :F] * (Z1 > 0)
        dW["e1"] += rnd(dZ1).T @ rnd(XE)
        dXE = rnd(dZ1) @ Wq["e1"]
        fl = g.nbr >= 0
        np.add.at(dh_prev, g.nbr[fl], dXE[fl, fe:fe + F])
        dh = dh_prev
    dZ0 = dh * (cache["z0"] > 0)
    dW["enc"] += rnd(dZ0).T @ rnd(g.u)
    return dW


def velocity_scale(gravity, dt_ad, u_ref):
    g = float(np.linalg.norm(np.asarray(gravity, dtype=np.float64)))
    return g * dt_ad if g > 0.0 else u_ref


def targets(dim, vel0, vel1, rho0_arr, rho1_arr, gravity, dt_ad, u_ref, rho0):
    """Normalised targets of one advection step (see the module header)."""
    T = np.zeros((vel0.shape[0], dim + 1))
    T[:, :dim] = (vel1 - vel0 - np.asarray(gravity)[:dim] * dt_ad) / velocity_scale(gravity, dt_ad, u_ref)
    T[:, dim] = S_RHO * (rho1_arr - rho0_arr) / rho0
    return T


@dataclass
class Adam:
    lr: float = 1e-3
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8


def adam_step(W, dW, m, v, t, opt: Adam):
    """One Adam update in place (t counts from 1)."""
    for k in W:
        m[k] = opt.b1 * m[k] + (1 - opt.b1) * dW[k]
        v[k] = opt.b2 * v[k] + (1 - opt.b2) * dW[k] ** 2
        mh = m[k] / (1 - opt.b1 ** t)
        vh = v[k] / (1 - opt.b2 ** t)
        W[k] = W[k] - opt.lr * mh / (np.sqrt(vh) + opt.eps)
