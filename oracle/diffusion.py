"""Plain FP64 CPU oracle of species diffusion on the fluid particles (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use this
module. It shares no code with the CUDA library.

The method (paper Sec. "Schemes for thermal and mass diffusion"), in the paper's order:

  * dC/dt = div(D grad C) (Eq. diffusion-eq) with a symmetric positive-definite tensor D,
    factored D = L L^T (Eq. chol).
  * The SPH form of the transformed Laplacian (Eq. grad-laplace):
        dC_i/dt = 2 sum_j (m_j/rho_j) (C_i - C_j) / (L~_ij e_ij)^2 * (1/r_ij) dW/dr_ij,
    with L~_ij the pair combination of the per-particle factors L~_i, D = L~_i^-1 L~_i^-T.
  * Time integration by a two-stage second-order Runge-Kutta scheme (Table tab:particle-dynamics:
    the diffusion process is integrated with RK2).

Readings where the paper is silent or inconsistent (the same readings the CUDA path takes):
  R13 One diffusion tensor per body. Then every L~_i equals L^-1, the pair combination of two
      equal factors is that factor (the printed combination L~_i L~_j/(L~_i + L~_j) is read as
      the harmonic mean, which it is up to the factor 2 that makes equal factors reproduce
      themselves), and the pair weight is 1/(L^-1 e)^2 = 1/(e^T D^-1 e); for isotropic
      D = kappa I it is kappa. Volumes are m_j/rho_j of the current state. The species lives
      on the fluid particles; wall particles carry none and exchange nothing (zero flux
      through walls). Pairs at zero distance contribute nothing (as reading R6 of the
      fluid oracle). The kernel-corrected form (Eq. grad-laplace-renormalize) is R31.
  R17 Per-particle diffusivity: D_i = s_i D with s_i > 0. Then L~_i = L^-1/sqrt(s_i), the
      harmonic combination of R13 gives L~_ij = L^-1 2/(sqrt(s_i) + sqrt(s_j)), and the pair
      weight is ((sqrt(s_i) + sqrt(s_j))/2)^2 / (e^T D^-1 e): the squared mean of the square
      roots, which equals s at a pair of equal factors.
  R14 RK2 is Heun's form: C* = C^n + dt f(C^n), C^{n+1} = (C^n + C* + dt f(C*))/2. The
      operator is linear and autonomous, so every two-stage second-order Runge-Kutta scheme
      gives the same C^{n+1} up to rounding.
  R15 For anisotropic D the printed operator is not consistent with div(D grad C): its
      continuum limit applied to a quadratic field with Hessian H is
      (d/|S|) int_S w(e) e^T H e dS over the unit sphere S (|S| its measure), with
      w(e) = 1/(e^T D^-1 e); it equals tr(D H) only when D is isotropic. The oracle
      computes the printed operator; the tests pin it against that closed-form limit.
  R32 Per-particle tensors of different shape, D_i = L_i L_i^T (Cholesky, Eq. chol), so
      L~_i = L_i^-1. The printed combination L~_i L~_j/(L~_i + L~_j), read as the harmonic
      mean of matrices (as R13 reads it for scalars), is L~_ij = 2 (L~_i^-1 + L~_j^-1)^-1
      = 2 (L_i + L_j)^-1, and the pair weight 1/(L~_ij e)^2 is r^2 / |M^-1 r|^2 with
      M = (L_i + L_j)/2. It is R13's 1/(e^T D^-1 e) when every D_i = D and R17's
      ((sqrt s_i + sqrt s_j)/2)^2 / (e^T D^-1 e) when D_i = s_i D, and it is symmetric in i
      and j, so the species is conserved.
  R31 The kernel-corrected form (Eq. grad-laplace-renormalize) as printed multiplies the
      matrix B0 by the scalar C and dots it with e.e = 1; read with the correction acting
      on the pair direction, e^T B0 e, and the two sides averaged: the pair weight of
      Eq. grad-laplace gains (e^T B0_i e + e^T B0_j e)/2. It reduces to Eq. grad-laplace for
      B0 = I, keeps both particles' matrices as printed, leaves constant fields at rest and,
      with a symmetric weight, conserves the species; the literal per-side product
      (e^T B0_i e C_i - e^T B0_j e C_j) moves a constant field wherever B0 varies. B0_i =
      (sum_j V_j (r_j - r_i) (x) grad_i W_ij)^-1 (Eq. sph-correctmatrix) over the species'
      pairs of the current configuration, V_j = m_j/rho_j; where that sum is singular (its
      determinant below 1e-6 (trace/d)^d, e.g. a particle with fewer than d neighbours
      spanning space) B0_i = I.

Parity pins: every function here is pinned by tests/test_diffusion_oracle.py (closed forms,
the analytic solution of a diffusing band, conservation, brute force). None is unpinned.
"""
from __future__ import annotations

import numpy as np

from oracle import wcsph as o


def tensor_inverse(D, dim: int) -> np.ndarray:
    """D^-1 of a symmetric positive-definite tensor, checked through its Cholesky factor
    (Eq. chol): L L^T = D with a positive diagonal exists only for SPD D."""
    D = np.asarray(D, dtype=np.float64).reshape(dim, dim)
    if not np.allclose(D, D.T, rtol=0.0, atol=0.0):
        raise ValueError("D must be symmetric")
    L = np.linalg.cholesky(D)           # raises for a tensor that is not positive definite
    Linv = np.linalg.inv(L)
    return Linv.T @ Linv                # (L L^T)^-1 = L^-T L^-1


def fluid_pairs(x: np.ndarray, prm: o.Params):
    """Directed fluid-fluid pairs of the neighbour set |r_i - r_j| < 2h, j != i."""
    I, J, _, _ = o.neighbour_sets(x, np.zeros((0, prm.dim)), prm)
    return I, J


def pair_scale(scale, I, J):
    """R17: pair factor of per-particle diffusivity factors s (D_i = s_i D). With
    L~_i = L^-1 / sqrt(s_i), the harmonic combination of R13 is L^-1 2/(sqrt(s_i) + sqrt(s_j)),
    so the pair weight gains ((sqrt(s_i) + sqrt(s_j))/2)^2."""
    if scale is None:
        return 1.0
    r = np.sqrt(np.asarray(scale, dtype=np.float64))
    return (0.5 * (r[I] + r[J])) ** 2


def correction_matrices(x, vol, I, J, prm: o.Params) -> np.ndarray:
    """R31: B0_i = (sum_j V_j (r_j - r_i) (x) grad_i W_ij)^-1 (Eq. sph-correctmatrix) over the
    directed pairs (I, J), the identity where the sum is singular."""
    n, d = x.shape[0], prm.dim
    rij = o.min_image(x[I] - x[J], prm.period)
    r = np.sqrt(np.sum(rij * rij, axis=1))
    ok = r > 0.0
    fw = np.zeros_like(r)
    fw[ok] = o.kernel_dW(r[ok], prm.h, d) / r[ok]                   # grad_i W_ij = fw r_ij
    outer = (vol[J] * fw)[:, None, None] * (-rij)[:, :, None] * rij[:, None, :]
    M = np.zeros((n, d, d))
    np.add.at(M, I, outer)
    B = np.broadcast_to(np.eye(d), (n, d, d)).copy()
    tr = np.trace(M, axis1=1, axis2=2) / d
    good = np.linalg.det(M) > 1e-6 * np.abs(tr) ** d
    B[good] = np.linalg.inv(M[good])
    return B


def tensor_factors(Dp, dim: int) -> np.ndarray:
    """R32: the Cholesky factor L_i of every particle's tensor D_i (Dp: (n, dim, dim)),
    each checked symmetric positive definite."""
    Dp = np.asarray(Dp, dtype=np.float64).reshape(-1, dim, dim)
    if not np.array_equal(Dp, np.swapaxes(Dp, 1, 2)):
        raise ValueError("every D_i must be symmetric")
    return np.linalg.cholesky(Dp)        # raises unless every D_i is positive definite


def diffusion_rate(x, C, vol, I, J, Dinv, prm: o.Params, scale=None, B=None, Lf=None) -> np.ndarray:
    """Eq. grad-laplace under R13 (and R17 with per-particle factors `scale`; with
    per-particle tensor factors Lf (n, d, d), R32, in place of Dinv; with the correction
    matrices B, Eq. grad-laplace-renormalize under R31): dC_i/dt for every fluid particle i."""
    rij = o.min_image(x[I] - x[J], prm.period)
    r2 = np.sum(rij * rij, axis=1)
    r = np.sqrt(r2)
    ok = r2 > 0.0
    fw = np.zeros_like(r)
    fw[ok] = o.kernel_dW(r[ok], prm.h, prm.dim) / r[ok]            # (1/r) dW/dr
    if Lf is None:
        quad = np.einsum("pa,ab,pb->p", rij, Dinv, rij)              # r^2 e^T D^-1 e
    else:                                                            # R32: |M^-1 r|^2, M = (L_i + L_j)/2
        M = 0.5 * (Lf[I] + Lf[J])
        y = np.linalg.solve(M, rij[:, :, None])[:, :, 0]
        quad = np.sum(y * y, axis=1)
    w = np.zeros_like(r)
    w[ok] = r2[ok] / quad[ok]                                        # 1/(L~ e)^2
    if B is not None:                                                # R31: (e^T B_i e + e^T B_j e)/2
        qi = np.einsum("pa,pab,pb->p", rij, B[I], rij)
        qj = np.einsum("pa,pab,pb->p", rij, B[J], rij)
        w[ok] = w[ok] * 0.5 * (qi[ok] + qj[ok]) / r2[ok]
    terms = 2.0 * vol[J] * (C[I] - C[J]) * fw * w * pair_scale(scale, I, J)
    out = np.zeros(x.shape[0])
    np.add.at(out, I, terms)
    return out


def rk2_step(x, C, vol, I, J, Dinv, dt: float, prm: o.Params, scale=None, B=None, Lf=None) -> np.ndarray:
    """One step of R14 (Heun)."""
    Cs = C + dt * diffusion_rate(x, C, vol, I, J, Dinv, prm, scale, B, Lf)
    return 0.5 * (C + Cs + dt * diffusion_rate(x, Cs, vol, I, J, Dinv, prm, scale, B, Lf))


def run(x, C, m, rho, D, dt: float, n_steps: int, prm: o.Params, scale=None, corrected=False,
        tensors=None) -> np.ndarray:
    """n_steps RK2 steps of the species C on static particles (positions x, masses m,
    densities rho; per-particle diffusivity factors `scale`, R17; per-particle tensors
    `tensors` (n, d, d) in place of D, R32, combined with `scale` as D_i = s_i tensors_i;
    the kernel-corrected form, R31, with `corrected`)."""
    x = np.asarray(x, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64).copy()
    vol = np.asarray(m, dtype=np.float64) / np.asarray(rho, dtype=np.float64)
    Dinv = tensor_inverse(D, prm.dim)
    I, J = fluid_pairs(x, prm)
    B = correction_matrices(x, vol, I, J, prm) if corrected else None
    Lf = None
    if tensors is not None:
        Lf = tensor_factors(tensors, prm.dim)
        if scale is not None:
            Lf = Lf * np.sqrt(np.asarray(scale, dtype=np.float64))[:, None, None]
            scale = None
    for _ in range(int(n_steps)):
        C = rk2_step(x, C, vol, I, J, Dinv, dt, prm, scale, B, Lf)
    return C
