"""Pins of the diffusion oracle (oracle/diffusion.py) against what the paper and the
mathematics fix: closed forms of the operator on quadratic fields, the closed-form
continuum limit of the printed anisotropic operator (reading R15), conservation, the
analytic solution of a diffusing band (the paper's first diffusion test, Sec. mass
diffusion), the amplification polynomial of the two-stage scheme, and brute force."""
import math

import numpy as np
import pytest

from oracle import diffusion as df
from oracle import wcsph as o
from paper_2010_12375_gb300 import workloads as wl


def _params(dim, h, dp, lo, hi, periodic):
    return o.Params(dim=dim, h=h, dp=dp, rho0=1.0, c0=1.0, cfl_ad=0.25, cfl_ac=0.6, u_ref=0.1,
                    nu=0.0, gravity=np.zeros(dim), lo=np.asarray(lo, float), hi=np.asarray(hi, float),
                    periodic=np.asarray(periodic, bool), free_surface=False)


def _centre_rate(dim, h_over_dp, D, H):
    """Rate at the centre particle of an unbounded lattice patch for C = x^T H x / 2."""
    dp = 1.0
    k = int(math.ceil(2 * h_over_dp)) + 1
    ax = np.arange(-k, k + 1, dtype=np.float64)
    X = np.stack([g.ravel() for g in np.meshgrid(*([ax] * dim), indexing="ij")], 1) * dp
    C = 0.5 * np.einsum("pa,ab,pb->p", X, H, X)
    i0 = int(np.nonzero(np.all(X == 0, axis=1))[0][0])
    J = np.array([j for j in range(X.shape[0]) if j != i0])
    I = np.full(J.size, i0)
    prm = _params(dim, h_over_dp * dp, dp, -np.full(dim, 100.0), np.full(dim, 100.0), [False] * dim)
    vol = np.full(X.shape[0], dp ** dim)
    return df.diffusion_rate(X, C, vol, I, J, df.tensor_inverse(D, dim), prm)[i0]


@pytest.mark.parametrize("dim", [2, 3])
def test_quadratic_isotropic_is_the_laplacian(dim):
    # div(kappa grad C) = kappa tr H exactly for a quadratic field; the lattice sum
    # converges to it as h/dp grows (1.3: 2.6 %, 4: < 2e-5)
    kappa = 0.7
    H = np.diag(np.arange(1.0, dim + 1.0))
    exact = kappa * np.trace(H)
    assert abs(_centre_rate(dim, 4.0, kappa * np.eye(dim), H) / exact - 1.0) < 2e-5
    assert abs(_centre_rate(dim, 1.3, kappa * np.eye(dim), H) / exact - 1.0) < 0.03


@pytest.mark.parametrize("H,limit", [
    # D = diag(4, 1) in 2D: w(theta) = 1/(cos^2/4 + sin^2); (2/2pi) int w e^T H e dtheta
    # with int cos^2/(A cos^2 + B sin^2) = 2 pi/(A + sqrt(AB)) and the sin^2 analogue
    (np.diag([2.0, 0.0]), 4.0 / (0.25 + 0.5)),
    (np.diag([0.0, 2.0]), 4.0 / (1.0 + 0.5)),
])
def test_anisotropic_printed_operator_limit(H, limit):
    # reading R15: the printed operator tends to (d/|S|) int w(e) e^T H e dS, not tr(D H)
    D = np.diag([4.0, 1.0])
    got = _centre_rate(2, 4.0, D, H)
    assert abs(got / limit - 1.0) < 5e-3
    assert abs(got / np.trace(D @ H) - 1.0) > 0.2                    # not div(D grad C)


def _jittered_box(dim, n, seed, periodic=True):
    rng = np.random.default_rng(seed)
    dp = 1.0 / n
    g = np.stack([a.ravel() for a in np.meshgrid(*([np.arange(n) + 0.5] * dim), indexing="ij")], 1) * dp
    x = g + rng.uniform(-0.2, 0.2, g.shape) * dp
    x = np.mod(x, 1.0) if periodic else x
    prm = _params(dim, 1.3 * dp, dp, np.zeros(dim), np.ones(dim), [periodic] * dim)
    return x, prm, rng


@pytest.mark.parametrize("dim", [2, 3])
def test_conservation_and_constant_field(dim):
    x, prm, rng = _jittered_box(dim, 12 if dim == 2 else 7, seed=3)
    n = x.shape[0]
    vol = prm.dp ** dim * rng.uniform(0.8, 1.2, n)
    C = rng.uniform(-1.0, 1.0, n)
    A = rng.normal(size=(dim, dim))
    D = A @ A.T + dim * np.eye(dim)                 # anisotropic, off-diagonal terms
    Dinv = df.tensor_inverse(D, dim)
    I, J = df.fluid_pairs(x, prm)
    r = df.diffusion_rate(x, C, vol, I, J, Dinv, prm)
    # antisymmetric pair exchange: sum_i V_i dC_i/dt = 0
    assert abs(np.sum(vol * r)) < 1e-12 * np.sum(np.abs(vol * r))
    assert np.all(df.diffusion_rate(x, np.full(n, 2.5), vol, I, J, Dinv, prm) == 0.0)


def test_brute_force_double_loop():
    # every pair term written out with plain loops on a tiny periodic box
    x, prm, rng = _jittered_box(2, 6, seed=11)
    n = x.shape[0]
    vol = prm.dp ** 2 * rng.uniform(0.8, 1.2, n)
    C = rng.uniform(0.0, 1.0, n)
    D = np.array([[2.0, 0.6], [0.6, 1.0]])
    Dinv = np.linalg.inv(D)
    I, J = df.fluid_pairs(x, prm)
    got = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(D, 2), prm)
    h = prm.h
    alpha = 7.0 / (4.0 * math.pi * h * h)
    want = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            d = x[i] - x[j]
            d -= np.round(d)                          # unit period
            r = math.hypot(d[0], d[1])
            if r >= 2 * h:
                continue
            q = r / h
            dW = alpha / h * (-5.0 * q) * (1 - q / 2) ** 3
            e = d / r
            w = 1.0 / float(e @ Dinv @ e)
            want[i] += 2.0 * vol[j] * (C[i] - C[j]) * w * dW / r
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))


def test_band_against_the_analytic_solution():
    # Sec. mass diffusion, first test: a band of pollutant (C = 1 for |x - 1/2| < a)
    # diffusing in 1D. On the unit-periodic axis the exact solution is the image sum
    # C = 1/2 sum_k [erf((a - (x - 1/2 + k))/s) + erf((a + (x - 1/2 + k))/s)], s = sqrt(4 kappa t).
    w = wl.diffusion_band(n=100, ny=8, kappa=1.0, a=0.1)
    prm = o.Params.from_problem(w)
    D = np.asarray(w.meta["D"])[:2, :2]
    dt = w.meta["dt"]
    steps = 150
    C = df.run(w.pos, w.meta["C0"], w.mass, w.rho, D, dt, steps, prm)
    s = math.sqrt(4.0 * 1.0 * dt * steps)
    xs = w.pos[:, 0] - 0.5
    exact = np.zeros_like(xs)
    for k in range(-2, 3):
        exact += 0.5 * (np.vectorize(math.erf)((0.1 - (xs + k)) / s) +
                        np.vectorize(math.erf)((0.1 + (xs + k)) / s))
    err = np.max(np.abs(C - exact))
    assert err < 1e-2
    # a planted factor-2 slip in the operator (kappa/2) is visible at this tolerance
    half = df.run(w.pos, w.meta["C0"], w.mass, w.rho, 0.5 * D, dt, steps, prm)
    assert np.max(np.abs(half - exact)) > 3e-2


def _sine_mode_rate(n, h_over_dp, kappa):
    dp = 1.0 / n
    g = np.stack([a.ravel() for a in np.meshgrid(np.arange(n) * dp, np.arange(n) * dp, indexing="ij")], 1)
    C0 = np.sin(2 * math.pi * g[:, 0])
    prm = _params(2, h_over_dp * dp, dp, [0, 0], [1, 1], [True, True])
    vol = np.full(g.shape[0], dp * dp)
    I, J = df.fluid_pairs(g, prm)
    Dinv = df.tensor_inverse(kappa * np.eye(2), 2)
    r = df.diffusion_rate(g, C0, vol, I, J, Dinv, prm)
    big = np.abs(C0) > 0.5
    lam = -r[big] / C0[big]
    assert np.ptp(lam) < 1e-9 * np.max(lam)          # an eigenvector of the operator
    return float(lam.mean()), (g, C0, vol, I, J, Dinv, prm)


def test_rk2_amplification_of_a_sine_mode():
    # a sine mode on a periodic lattice is an eigenvector of the linear operator, so one
    # two-stage second-order step multiplies it by 1 - z + z^2/2 with z = lambda dt
    kappa, k2 = 0.3, (2 * math.pi) ** 2
    lam, (g, C0, vol, I, J, Dinv, prm) = _sine_mode_rate(40, 1.3, kappa)
    assert abs(lam / (kappa * k2) - 1.0) < 0.03
    dt = 0.1 * prm.h ** 2 / kappa
    C = C0.copy()
    for _ in range(5):
        C = df.rk2_step(g, C, vol, I, J, Dinv, dt, prm)
    z = lam * dt
    np.testing.assert_allclose(C, (1 - z + z * z / 2) ** 5 * C0, rtol=0, atol=1e-12)


def test_sine_mode_rate_converges_at_second_order():
    # at fixed h/dp = 3 the rate tends to kappa k^2 with an error of order (k h)^2
    kappa, k2 = 0.3, (2 * math.pi) ** 2
    e40 = abs(_sine_mode_rate(40, 3.0, kappa)[0] / (kappa * k2) - 1.0)
    e80 = abs(_sine_mode_rate(80, 3.0, kappa)[0] / (kappa * k2) - 1.0)
    assert e40 < 0.02 and 3.5 < e40 / e80 < 4.5


def test_tensor_inverse_rejects_bad_tensors():
    with pytest.raises(ValueError):
        df.tensor_inverse([[1.0, 0.2], [0.0, 1.0]], 2)          # not symmetric
    with pytest.raises(np.linalg.LinAlgError):
        df.tensor_inverse([[1.0, 2.0], [2.0, 1.0]], 2)          # indefinite
    D = np.array([[3.0, 1.0], [1.0, 2.0]])
    np.testing.assert_allclose(df.tensor_inverse(D, 2) @ D, np.eye(2), atol=1e-14)


def _centre_rate_scaled(h_over_dp, C_of, s_of, x0):
    """Rate at the lattice point nearest x0 (2D, isotropic D = I) with per-particle
    factors s(x) and field C(x)."""
    dp = 1.0
    k = int(math.ceil(2 * h_over_dp)) + 1
    ax = np.arange(-k, k + 1, dtype=np.float64)
    X = np.stack([g.ravel() for g in np.meshgrid(ax, ax, indexing="ij")], 1) * dp + np.asarray(x0)
    i0 = int(np.argmin(np.sum((X - np.asarray(x0)) ** 2, axis=1)))
    J = np.array([j for j in range(X.shape[0]) if j != i0])
    I = np.full(J.size, i0)
    prm = _params(2, h_over_dp * dp, dp, -np.full(2, 100.0), np.full(2, 100.0), [False, False])
    vol = np.full(X.shape[0], dp * dp)
    return df.diffusion_rate(X, C_of(X), vol, I, J, np.eye(2), prm, scale=s_of(X))[i0]


def test_per_particle_diffusivity_gives_the_variable_coefficient_operator():
    # reading R17: with D_i = s_i I the operator tends to div(s grad C) = s lap C + grad s . grad C
    # C = x^2 + y^2 / 2, s = 2 + 0.05 x + 0.02 y at x0 = (3, -2):
    # lap C = 3, grad C = (6, -2), grad s = (0.05, 0.02) -> s lap C + grad s . grad C
    C_of = lambda X: X[:, 0] ** 2 + 0.5 * X[:, 1] ** 2
    s_of = lambda X: 2.0 + 0.05 * X[:, 0] + 0.02 * X[:, 1]
    x0 = (3.0, -2.0)
    exact = (2.0 + 0.15 - 0.04) * 3.0 + (0.05 * 6.0 - 0.02 * 2.0)
    got = _centre_rate_scaled(4.0, C_of, s_of, x0)
    assert abs(got / exact - 1.0) < 1e-3
    # a one-sided factor (s_i alone) drops the grad s . grad C term and fails
    one_sided = lambda X: np.full(X.shape[0], 2.0 + 0.15 - 0.04)
    assert abs(_centre_rate_scaled(4.0, C_of, one_sided, x0) / exact - 1.0) > 0.03


def test_uniform_factor_scales_the_tensor():
    x, prm, rng = _jittered_box(2, 10, seed=5)
    n = x.shape[0]
    vol = prm.dp ** 2 * rng.uniform(0.9, 1.1, n)
    C = rng.uniform(0.0, 1.0, n)
    D = np.array([[1.5, 0.3], [0.3, 0.8]])
    I, J = df.fluid_pairs(x, prm)
    a = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(2.5 * D, 2), prm)
    b = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(D, 2), prm, scale=np.full(n, 2.5))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.max(np.abs(a)))
    s = rng.uniform(0.5, 2.0, n)                    # conservation with varying factors
    r = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(D, 2), prm, scale=s)
    assert abs(np.sum(vol * r)) < 1e-12 * np.sum(np.abs(vol * r))


def test_anisotropic_printed_operator_limit_3d():
    # reading R15 in 3D: D = diag(4, 4, 1), C = z^2. With mu = cos(theta) and A = 1/4, B = 1,
    # w = 1/(A (1 - mu^2) + B mu^2) and (3/4pi) int w 2 mu^2 dS = 3 int_-1^1 mu^2/(A + (B-A) mu^2) dmu
    # = 3 (2 - (2/k) atan k)/(A k^2), k^2 = (B - A)/A; tr(D H) would be 2
    A, B = 0.25, 1.0
    k = math.sqrt((B - A) / A)
    limit = 3.0 * (2.0 - (2.0 / k) * math.atan(k)) / (A * k * k)
    got = _centre_rate(3, 4.0, np.diag([4.0, 4.0, 1.0]), np.diag([0.0, 0.0, 2.0]))
    assert abs(got / limit - 1.0) < 2e-3
    assert abs(got / 2.0 - 1.0) > 0.3


# ---- kernel-corrected form (Eq. grad-laplace-renormalize, reading R31) ------------------------

def _patch_operator(n=30):
    w = wl.diffusion_patch(n)
    prm = o.Params.from_problem(w)
    x, vol = w.pos, w.mass / w.rho
    I, J = df.fluid_pairs(x, prm)
    return w, prm, x, vol, I, J, df.correction_matrices(x, vol, I, J, prm)


def test_correction_matrix_is_the_inverse_lattice_moment():
    # written out for one particle: B0 (sum_j V_j (r_j - r_i) (x) grad_i W_ij) = I
    w, prm, x, vol, I, J, B = _patch_operator(20)
    for i in (0, 45, 210):
        M = np.zeros((2, 2))
        for j in J[I == i]:
            r = x[i] - x[j]
            d = np.linalg.norm(r)
            M += vol[j] * np.outer(-r, o.kernel_dW(d, prm.h, 2) / d * r)
        assert np.allclose(B[i] @ M, np.eye(2), atol=1e-12)
    # a particle with no neighbours keeps the identity
    B1 = df.correction_matrices(np.array([[0.5, 0.5], [0.9, 0.9]]), np.ones(2), np.zeros(0, int), np.zeros(0, int), prm)
    assert np.array_equal(B1, np.broadcast_to(np.eye(2), (2, 2, 2)))


def test_corrected_form_with_identity_is_the_plain_form():
    w, prm, x, vol, I, J, B = _patch_operator()
    C = np.random.default_rng(3).random(len(x))
    eye = np.broadcast_to(np.eye(2), B.shape)
    plain = df.diffusion_rate(x, C, vol, I, J, np.eye(2), prm)
    assert np.allclose(df.diffusion_rate(x, C, vol, I, J, np.eye(2), prm, None, eye), plain, rtol=1e-13, atol=0)


def test_corrected_form_removes_the_lattice_error_at_second_order():
    # sin 2 pi x sin 2 pi y on the unit-periodic lattice: the plain form keeps the lattice-sum
    # error (3.2 % at 40^2, 2.7 % at 80^2); the corrected one converges at second order
    # (0.58 %, 0.145 %)
    errs = {}
    for n in (40, 80):
        w = wl.diffusion_band(n, ny=n)
        prm = o.Params.from_problem(w)
        x, vol = w.pos, w.mass / w.rho
        I, J = df.fluid_pairs(x, prm)
        B = df.correction_matrices(x, vol, I, J, prm)
        C = np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1])
        exact = -8.0 * np.pi ** 2 * C
        for key, Bm in (("plain", None), ("corrected", B)):
            L = df.diffusion_rate(x, C, vol, I, J, np.eye(2), prm, None, Bm)
            errs[key, n] = np.linalg.norm(L - exact) / np.linalg.norm(exact)
    assert errs["plain", 40] > 0.02 and errs["plain", 80] > 0.02
    assert errs["corrected", 40] < 0.01 and errs["corrected", 80] < 0.002
    assert errs["corrected", 40] / errs["corrected", 80] > 3.5


def test_corrected_form_on_free_edges_conserves_and_is_exact_inside():
    w, prm, x, vol, I, J, B = _patch_operator()
    assert np.abs(B - B[len(B) // 2]).max() > 0.5                    # B0 varies near the edges
    one = np.ones(len(x))
    assert np.abs(df.diffusion_rate(x, one, vol, I, J, np.eye(2), prm, None, B)).max() == 0.0
    C = np.random.default_rng(5).random(len(x))
    L = df.diffusion_rate(x, C, vol, I, J, np.eye(2), prm, None, B)
    assert abs(np.sum(vol * L)) < 1e-12 * np.sum(np.abs(vol * L))
    edge = np.minimum.reduce([x[:, 0], x[:, 1], 1 - x[:, 0], 1 - x[:, 1]])
    inner = edge > 2 * prm.h + w.dp
    q = x[:, 0] ** 2 + x[:, 1] ** 2                                   # Laplacian 4
    Lq = df.diffusion_rate(x, q, vol, I, J, np.eye(2), prm, None, B)
    Lp = df.diffusion_rate(x, q, vol, I, J, np.eye(2), prm)
    assert np.abs(Lq[inner] - 4.0).max() < 1e-9 and np.abs(Lp[inner] - 4.0).min() > 0.1


def test_corrected_form_planted_mistake_moves_a_constant_field():
    # the literal per-side product (e^T B_i e C_i - e^T B_j e C_j) is what R31 rejects: it
    # gives a constant field a non-zero rate wherever B0 varies
    w, prm, x, vol, I, J, B = _patch_operator()
    rij = x[I] - x[J]
    r2 = np.sum(rij * rij, axis=1)
    qi = np.einsum("pa,pab,pb->p", rij, B[I], rij) / r2
    qj = np.einsum("pa,pab,pb->p", rij, B[J], rij) / r2
    fw = o.kernel_dW(np.sqrt(r2), prm.h, 2) / np.sqrt(r2)
    literal = np.zeros(len(x))
    np.add.at(literal, I, 2.0 * vol[J] * (qi - qj) * fw)             # C = 1
    assert np.abs(literal).max() > 100.0


# ---- per-particle tensors of different shape (reading R32) -----------------------------------

def _box_operator(n=24, seed=4):
    w = wl.periodic_box(2, n=n, seed=seed, vel_amp=0.0)
    prm = o.Params.from_problem(w)
    x, vol = w.pos, w.mass / w.rho
    I, J = df.fluid_pairs(x, prm)
    return w, prm, x, vol, I, J


def _random_spd(rng, n, d):
    A = rng.normal(size=(n, d, d))
    return A @ np.swapaxes(A, 1, 2) + 0.5 * np.eye(d)


def test_equal_tensors_are_the_single_tensor_operator():
    w, prm, x, vol, I, J = _box_operator()
    D = np.array([[2.0, 0.6], [0.6, 1.0]])
    C = np.random.default_rng(1).random(len(x))
    Lf = df.tensor_factors(np.broadcast_to(D, (len(x), 2, 2)), 2)
    a = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(D, 2), prm)
    b = df.diffusion_rate(x, C, vol, I, J, None, prm, Lf=Lf)
    assert np.allclose(b, a, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_scaled_tensors_are_the_per_particle_factor_operator():
    # D_i = s_i D gives R17's ((sqrt s_i + sqrt s_j)/2)^2 / (e^T D^-1 e)
    w, prm, x, vol, I, J = _box_operator()
    rng = np.random.default_rng(2)
    D = np.array([[1.5, -0.4], [-0.4, 0.8]])
    s = rng.uniform(0.5, 2.0, len(x))
    C = rng.random(len(x))
    Lf = df.tensor_factors(s[:, None, None] * D, 2)
    a = df.diffusion_rate(x, C, vol, I, J, df.tensor_inverse(D, 2), prm, scale=s)
    b = df.diffusion_rate(x, C, vol, I, J, None, prm, Lf=Lf)
    assert np.allclose(b, a, rtol=1e-11, atol=1e-11 * np.abs(a).max())


def test_tensors_of_different_shape_conserve_and_keep_constants():
    w, prm, x, vol, I, J = _box_operator()
    rng = np.random.default_rng(3)
    Lf = df.tensor_factors(_random_spd(rng, len(x), 2), 2)
    C = rng.random(len(x))
    L = df.diffusion_rate(x, C, vol, I, J, None, prm, Lf=Lf)
    assert abs(np.sum(vol * L)) < 1e-12 * np.sum(np.abs(vol * L))
    assert np.abs(df.diffusion_rate(x, np.ones(len(x)), vol, I, J, None, prm, Lf=Lf)).max() == 0.0
    with pytest.raises(np.linalg.LinAlgError):                        # not positive definite
        df.tensor_factors(np.broadcast_to(np.diag([1.0, -1.0]), (3, 2, 2)), 2)


def test_tensors_planted_mistake_breaks_conservation():
    # taking only particle i's factor (M = L_i) makes the pair weight one-sided: the species
    # is no longer conserved
    w, prm, x, vol, I, J = _box_operator()
    rng = np.random.default_rng(3)
    Lf = df.tensor_factors(_random_spd(rng, len(x), 2), 2)
    C = rng.random(len(x))
    rij = o.min_image(x[I] - x[J], prm.period)
    y = np.linalg.solve(Lf[I], rij[:, :, None])[:, :, 0]
    r2 = np.sum(rij * rij, axis=1)
    r = np.sqrt(r2)
    terms = 2.0 * vol[J] * (C[I] - C[J]) * o.kernel_dW(r, prm.h, 2) / r * r2 / np.sum(y * y, axis=1)
    L = np.zeros(len(x))
    np.add.at(L, I, terms)
    assert abs(np.sum(vol * L)) > 1e-6 * np.sum(np.abs(vol * L))
