"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

The paper prints no numeric worked example (its figures are not available and
its text gives only speed-up ratios), so each oracle routine is pinned by:
closed forms for n = 1 and n = 2, exact rational arithmetic on tiny inputs,
LAPACK routines for the special cases they solve, the l -> 0 and l -> infinity
limits (Sherman-Morrison), invariants of Eqs. 3-4, central finite differences
of Eq. 5, and the defining properties of Adam.  None of these re-types the
oracle's own loops.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial.distance import cdist

from paper_2505_00136_gb300 import datagen as dg
from _util import rel, max_rel

import oracle as oracle_mod

HYP = (1.0, 1.0, 0.1)


def small_set(n=48, m=16, d=8, seed=1001):
    return dg.msd_dataset(n, m, d, seed)


# --------------------------------------------------------------------------- Eq. 2

def test_kernel_diagonal_exact_and_symmetric(orc):
    X, _, _, _ = small_set()
    K = orc.cov_train(X, (0.7, 1.3, 0.2))
    assert np.all(np.diag(K) == 1.3 + 0.2)            # r = 0 -> nu + sigma^2 exactly
    assert np.array_equal(K, K.T)


def test_kernel_one_dimensional_closed_form(orc):
    h, l, nu = 0.5, 1.7, 2.5                            # grid spacing exact in binary
    X = (np.arange(12) * h).reshape(-1, 1)
    idx = np.arange(12)
    expect = nu * np.exp(-((idx[:, None] - idx[None, :]) * h) ** 2 / (2 * l * l))
    assert max_rel(orc.se_cross(X, X, l, nu), expect) < 4e-16


def test_kernel_matches_library_distances_and_is_translation_invariant(orc):
    X, _, Xs, _ = small_set(d=5)
    l, nu = 0.9, 1.1
    expect = nu * np.exp(-cdist(Xs, X, "sqeuclidean") / (2 * l * l))
    assert max_rel(orc.se_cross(Xs, X, l, nu), expect) < 1e-13
    shifted = orc.se_cross(Xs + 0.25, X + 0.25, l, nu)
    assert max_rel(shifted, orc.se_cross(Xs, X, l, nu)) < 1e-13


# --------------------------------------------------------------------------- Cholesky, solves

def test_cholesky_against_lapack_and_reconstruction(orc):
    X, _, _, _ = small_set(n=96)
    K = orc.cov_train(X, HYP)
    L = orc.cholesky(K)
    assert np.all(np.triu(L, 1) == 0.0)
    assert rel(L, np.linalg.cholesky(K)) < 1e-13
    assert np.linalg.norm(L @ L.T - K) / np.linalg.norm(K) < 96 * 2.2e-16 * 10


def test_cholesky_reports_first_non_positive_pivot(orc):
    X = np.zeros((6, 3))                                # identical rows, sigma^2 = 0: K = 11^T exactly
    K = orc.cov_train(X, (1.0, 1.0, 0.0))
    with pytest.raises(oracle_mod.OracleNotPD) as e:
        orc.cholesky(K)
    assert e.value.row == 1                            # pivot 1 - 1*1 = 0 exactly
    A = np.diag([4.0, 9.0, -1.0, 2.0])
    with pytest.raises(oracle_mod.OracleNotPD) as e:
        orc.cholesky(A)
    assert e.value.row == 2


def test_triangular_solves_and_inverses_against_lapack(orc):
    X, y, _, _ = small_set(n=64)
    K = orc.cov_train(X, HYP)
    L = orc.cholesky(K)
    assert rel(orc.forward(L, y), sla.solve_triangular(L, y, lower=True)) < 1e-13
    assert rel(orc.backward(L, y), sla.solve_triangular(L.T, y, lower=False)) < 1e-13
    assert rel(orc.tri_inverse(L), sla.solve_triangular(L, np.eye(64), lower=True)) < 1e-13
    Kinv = orc.chol_inverse(L)
    assert rel(Kinv, sla.cho_solve((L, True), np.eye(64))) < 1e-12
    assert np.linalg.norm(Kinv @ K - np.eye(64)) < 1e-10


# --------------------------------------------------------------------------- closed forms

def test_n1_closed_forms(orc):
    l, nu, s2 = 0.8, 1.7, 0.3
    X = np.array([[0.2, -0.4]])
    y = np.array([0.9])
    xs = np.array([[0.5, 0.1]])
    a = nu + s2
    k = nu * np.exp(-((0.5 - 0.2) ** 2 + (0.1 + 0.4) ** 2) / (2 * l * l))
    mu, va, cv = orc.predict(X, y, xs, (l, nu, s2), cov=True)
    assert abs(mu[0] - k * 0.9 / a) < 1e-15
    assert abs(va[0] - (nu - k * k / a)) < 1e-15
    assert abs(cv[0, 0] - va[0]) < 1e-15
    f_expect = 0.5 * np.log(2 * np.pi * a) + 0.9 ** 2 / (2 * a)
    f, g = orc.nlml_grad(X, y, (l, nu, s2))
    assert abs(f - f_expect) < 1e-14
    common = 1.0 / (2 * a) - 0.9 ** 2 / (2 * a * a)     # dNLML/da
    assert abs(g[0]) == 0.0                              # r = 0: no length-scale dependence
    assert abs(g[1] - nu * common) < 1e-15
    assert abs(g[2] - s2 * common) < 1e-15


def test_n2_closed_forms(orc):
    l, nu, s2 = 1.3, 0.9, 0.2
    X = np.array([[0.0, 0.5], [0.75, -0.25]])
    y = np.array([0.4, -1.1])
    xs = np.array([[0.25, 0.25]])
    r2 = 0.75 ** 2 + 0.75 ** 2
    a, c = nu + s2, nu * np.exp(-r2 / (2 * l * l))
    det = a * a - c * c
    Kinv = np.array([[a, -c], [-c, a]]) / det
    alpha = Kinv @ y
    kh = nu * np.exp(-np.array([0.25 ** 2 + 0.25 ** 2, 0.5 ** 2 + 0.5 ** 2]) / (2 * l * l))
    mu, va, _ = orc.predict(X, y, xs, (l, nu, s2))
    assert abs(mu[0] - kh @ alpha) < 1e-14
    assert abs(va[0] - (nu - kh @ Kinv @ kh)) < 1e-14
    f = orc.nlml(X, y, (l, nu, s2))
    assert abs(f - (0.5 * y @ alpha + 0.5 * np.log(det) + np.log(2 * np.pi))) < 1e-14
    # gradient: dK/dlog l has only the off-diagonal c r2/l^2, dK/dlog nu = K_f, dK/dlog s2 = s2 I
    W = Kinv - np.outer(alpha, alpha)
    g_expect = [0.5 * 2 * W[0, 1] * c * r2 / (l * l),
                0.5 * (W[0, 0] * nu + W[1, 1] * nu + 2 * W[0, 1] * c),
                0.5 * s2 * (W[0, 0] + W[1, 1])]
    _, g = orc.nlml_grad(X, y, (l, nu, s2))
    assert max_rel(g, g_expect) < 1e-12


def _exact_solve(A, b):
    """Gauss-Jordan in exact rational arithmetic."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][k] - f * M[c][k] for k in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


def _exact_det(A):
    n = len(A)
    M = [list(r) for r in A]
    det = Fraction(1)
    for c in range(n):
        for r in range(c + 1, n):
            f = M[r][c] / M[c][c]
            M[r] = [M[r][k] - f * M[c][k] for k in range(n)]
        det *= M[c][c]
    return det


def test_tiny_problem_against_exact_rational_arithmetic(orc):
    X, y, Xs, _ = small_set(n=6, m=3, d=3, seed=77)
    hyp = (0.9, 1.2, 0.05)
    K = orc.cov_train(X, hyp)                          # float entries, taken as exact rationals
    Kc = orc.se_cross(Xs, X, hyp[0], hyp[1])
    KF = [[Fraction(v) for v in row] for row in K]
    yF = [Fraction(v) for v in y]
    alpha = _exact_solve(KF, yF)
    mu, va, _ = orc.predict(X, y, Xs, hyp)
    for i in range(3):
        kF = [Fraction(v) for v in Kc[i]]
        mean_i = sum(a * b for a, b in zip(kF, alpha))
        q = sum(a * b for a, b in zip(kF, _exact_solve(KF, kF)))
        assert abs(mu[i] - float(mean_i)) < 1e-14 * max(1.0, abs(float(mean_i)))
        assert abs(va[i] - float(Fraction(hyp[1]) - q)) < 1e-14
    fit = float(sum(a * b for a, b in zip(yF, alpha)))
    logdet = np.log(float(_exact_det(KF)))
    f_expect = 0.5 * fit + 0.5 * logdet + 3 * np.log(2 * np.pi)
    assert abs(orc.nlml(X, y, hyp) - f_expect) < 1e-13 * abs(f_expect)


# --------------------------------------------------------------------------- limits

def test_short_length_scale_limit(orc):
    X = dg.random_points(40, 4, seed=3)
    Xs = dg.random_points(10, 4, seed=4)
    y = dg.uniform(5, 0, 40, -1, 1)
    nu, s2 = 1.4, 0.3
    hyp = (1e-3, nu, s2)                               # exp(-r^2/2l^2) underflows to 0
    mu, va, cv = orc.predict(X, y, Xs, hyp, cov=True)
    assert np.all(mu == 0.0) and np.all(va == nu)
    assert np.array_equal(cv, np.diag(np.full(10, nu)))
    f = orc.nlml(X, y, hyp)
    f_expect = 0.5 * 40 * np.log(2 * np.pi * (nu + s2)) + y @ y / (2 * (nu + s2))
    assert abs(f - f_expect) < 1e-13 * abs(f_expect)


def test_long_length_scale_limit_sherman_morrison(orc):
    X = dg.random_points(30, 3, seed=8)
    Xs = dg.random_points(5, 3, seed=9)
    y = dg.uniform(10, 0, 30, -1, 1)
    nu, s2, n = 0.8, 0.25, 30
    hyp = (1e8, nu, s2)                                # K_f -> nu 11^T
    one = np.ones(n)
    alpha = (y - nu * one * (one @ y) / (s2 + n * nu)) / s2          # Sherman-Morrison
    mu, va, _ = orc.predict(X, y, Xs, hyp)
    assert max_rel(mu, np.full(5, nu * one @ alpha), 1e-3) < 1e-9
    var_expect = nu - nu * nu * n / (s2 + n * nu)      # 1^T K^{-1} 1 = n/(s2 + n nu)
    assert np.all(np.abs(va - var_expect) < 1e-9)
    logdet = (n - 1) * np.log(s2) + np.log(s2 + n * nu)
    f_expect = 0.5 * y @ alpha + 0.5 * logdet + 0.5 * n * np.log(2 * np.pi)
    assert abs(orc.nlml(X, y, hyp) - f_expect) < 1e-10 * abs(f_expect)


# --------------------------------------------------------------------------- invariants

def test_variance_bounds_and_full_covariance_consistency(orc):
    X, y, Xs, _ = small_set(n=80, m=24)
    hyp = (0.9, 1.3, 0.1)
    for noisy in (False, True):
        mu, va, cv = orc.predict(X, y, Xs, hyp, noisy=noisy, cov=True)
        upper = hyp[1] + (hyp[2] if noisy else 0.0)
        assert np.all(va >= 0) and np.all(va <= upper)
        assert np.array_equal(np.diag(cv), va) or max_rel(np.diag(cv), va) < 1e-14
        assert np.allclose(cv, cv.T, rtol=0, atol=1e-15)
        assert np.linalg.eigvalsh(cv).min() > -1e-12
    # the noisy variant adds exactly sigma^2
    _, v0, _ = orc.predict(X, y, Xs, hyp, noisy=False)
    _, v1, _ = orc.predict(X, y, Xs, hyp, noisy=True)
    assert np.allclose(v1 - v0, hyp[2], rtol=0, atol=1e-15)


def test_mean_interpolates_as_noise_vanishes(orc):
    X = dg.random_points(20, 2, seed=11)
    y = np.sin(3 * X[:, 0]) + X[:, 1]
    mu, va, _ = orc.predict(X, y, X, (0.5, 1.0, 1e-10))
    assert np.max(np.abs(mu - y)) < 1e-6
    assert np.max(np.abs(va)) < 1e-6


def test_permutation_invariance_and_two_mean_forms(orc):
    X, y, Xs, _ = small_set(n=50, m=12)
    perm = np.random.default_rng(0).permutation(50)
    a = orc.predict(X, y, Xs, HYP, cov=True)
    b = orc.predict(X[perm], y[perm], Xs, HYP, cov=True)
    for u, v in zip(a, b):
        assert rel(u, v) < 1e-12
    assert abs(orc.nlml(X, y, HYP) - orc.nlml(X[perm], y[perm], HYP)) < 1e-12
    # K_{Z*,Z} alpha == V^T beta with V = L^{-1} K_{Z*,Z}^T, beta = L^{-1} y
    L = orc.cholesky(orc.cov_train(X, HYP))
    beta = orc.forward(L, y)
    Kc = orc.se_cross(Xs, X, HYP[0], HYP[1])
    V = np.stack([orc.forward(L, Kc[i]) for i in range(12)], axis=1)
    assert rel(V.T @ beta, a[0]) < 1e-13


def test_predictive_quantities_against_lapack(orc):
    X, y, Xs, _ = small_set(n=128, m=32)
    hyp = (1.1, 0.8, 0.15)
    K = orc.cov_train(X, hyp)
    Kc = orc.se_cross(Xs, X, hyp[0], hyp[1])
    Kss = orc.se_cross(Xs, Xs, hyp[0], hyp[1])
    cf = sla.cho_factor(K, lower=True)
    mu_e = Kc @ sla.cho_solve(cf, y)
    cov_e = Kss - Kc @ sla.cho_solve(cf, Kc.T)
    mu, va, cv = orc.predict(X, y, Xs, hyp, cov=True)
    assert rel(mu, mu_e) < 1e-12
    assert rel(cv, cov_e) < 1e-11
    sign, logdet = np.linalg.slogdet(K)
    f_e = 0.5 * y @ sla.cho_solve(cf, y) + 0.5 * logdet + 64 * np.log(2 * np.pi)
    assert abs(orc.nlml(X, y, hyp) - f_e) < 1e-12 * abs(f_e)


# --------------------------------------------------------------------------- gradient, Adam

@pytest.mark.parametrize("hyp", [(1.0, 1.0, 0.1), (0.6, 2.0, 0.03), (2.2, 0.5, 0.4)])
def test_gradient_against_central_differences(orc, hyp):
    X, y, _, _ = small_set(n=40, d=4, seed=1004)
    f, g = orc.nlml_grad(X, y, hyp)
    assert abs(f - orc.nlml(X, y, hyp)) == 0.0
    h = 1e-5
    th = np.log(hyp)
    fd = np.empty(3)
    for p in range(3):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (orc.nlml(X, y, np.exp(tp)) - orc.nlml(X, y, np.exp(tm))) / (2 * h)
    assert max_rel(g, fd, floor=1e-8 * np.linalg.norm(fd)) < 1e-7


def test_adam_constant_gradient_steps_are_exactly_lr(orc):
    # With a constant gradient the bias-corrected moments equal g and g^2, so every
    # step moves each trainable coordinate by lr * g / (|g| + eps).
    g = np.array([0.3, -2.0, 5e-3])
    th, mo, ve = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 8):
        prev = th
        th, mo, ve = orc.adam(th, mo, ve, g, t, lr=0.05)
        assert max_rel(th - prev, -0.05 * g / (np.abs(g) + 1e-8)) < 1e-12


def test_adam_mask_and_scale_invariance(orc):
    g1 = np.array([0.3, -2.0, 1.5])
    g2 = np.array([-0.1, 0.7, 0.2])
    th_a = orc.adam(np.ones(3), np.zeros(3), np.zeros(3), g1, 1, eps=0.0)
    th_a = orc.adam(*th_a, g2, 2, eps=0.0)[0]
    th_b = orc.adam(np.ones(3), np.zeros(3), np.zeros(3), 1e3 * g1, 1, eps=0.0)
    th_b = orc.adam(*th_b, 1e3 * g2, 2, eps=0.0)[0]
    assert max_rel(th_a, th_b) < 1e-14
    th_m = orc.adam(np.ones(3), np.zeros(3), np.zeros(3), g1, 1, trainable=(1, 0, 1))[0]
    assert th_m[1] == 1.0 and th_m[0] != 1.0 and th_m[2] != 1.0


def test_optimize_matches_torch_adam_on_log_parameters(orc):
    """orc_optimize against an independent Adam (torch.optim.Adam, float64) acting
    on log theta, each step fed the oracle's own gradient (pinned above by finite
    differences): the NLML history and the final hyperparameters agree step by
    step.  Adam on the natural scale, a dropped bias correction or a wrong sign
    would each move the trajectory by far more than the bound."""
    torch = pytest.importorskip("torch")
    X, y, _, _ = small_set(n=48, d=4, seed=1006)
    hyp0, steps, lr = (0.9, 1.2, 0.07), 25, 0.1
    h_o, hist_o = orc.optimize(X, y, hyp0, steps=steps, lr=lr)
    th = torch.tensor(np.log(hyp0), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([th], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    hist = []
    for _ in range(steps):
        f, g = orc.nlml_grad(X, y, np.exp(th.detach().numpy()))
        hist.append(f)
        opt.zero_grad()
        th.grad = torch.from_numpy(g.copy())
        opt.step()
    assert max_rel(hist, hist_o) < 1e-10
    assert max_rel(np.exp(th.detach().numpy()), h_o) < 1e-10
    assert hist_o[-1] < hist_o[0]


def test_optimize_history_and_descent(orc):
    X, y, _, _ = small_set(n=64, d=4, seed=1004)
    h, hist = orc.optimize(X, y, HYP, steps=30, lr=0.1)
    assert hist[0] == orc.nlml(X, y, HYP)
    assert hist[-1] < hist[0]
    assert orc.nlml(X, y, h) < hist[0]


# --------------------------------------------------------------------------- learned-initialiser pieces

def test_summary_against_numpy_statistics(orc):
    X, y, _, _ = dg.msd_dataset(300, 0, 12, seed=5)
    om = dg.rff_frequencies()
    s = orc.summary(X, y, om)
    sd = np.sort(X.std(axis=0))[::-1]
    assert max_rel(s[:12], sd) < 1e-12 and np.all(s[12:32] == 0)
    yc = y - y.mean()
    ac = np.correlate(yc, yc, "full")[len(y) - 1:] / (yc @ yc)
    assert max_rel(s[32:48], ac[1:17], floor=1e-3) < 1e-11
    const = orc.summary(X, np.full(300, 0.375), om)
    assert max_rel(const[48::2], np.cos(om * 0.375)) < 1e-14
    assert max_rel(const[49::2], np.sin(om * 0.375), floor=1e-12) < 1e-13
    perm = np.random.default_rng(1).permutation(300)
    sp = orc.summary(X[perm], y[perm], om)
    assert rel(sp[:32], s[:32]) < 1e-14 and rel(sp[48:], s[48:]) < 1e-13
    wide = orc.summary(np.tile(X, (1, 4)), y, om)       # 48 regressors: truncated to 32
    assert max_rel(wide[:32], np.sort(np.tile(X, (1, 4)).std(axis=0))[::-1][:32]) < 1e-12


def _mlp_layers(W):
    o = 0
    shapes = [(256, 64), (256,), (256, 256), (256,), (3, 256), (3,)]
    out = []
    for sh in shapes:
        k = int(np.prod(sh))
        out.append(W[o:o + k].reshape(sh))
        o += k
    return out


def test_mlp_forward_against_matrix_products_and_backward_against_fd(orc):
    rng = np.random.default_rng(2)
    W = rng.normal(0, 0.1, oracle_mod.Oracle.MLP_NPARAM)
    S = rng.normal(0, 1, (5, 64))
    T = rng.normal(0, 1, (5, 3))
    W1, b1, W2, b2, W3, b3 = _mlp_layers(W)
    h1 = np.maximum(S @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    out = h2 @ W3.T + b3
    assert rel(orc.mlp_forward(W, S), out) < 1e-13
    loss, g = orc.mlp_loss_grad(W, S, T)
    assert abs(loss - np.mean((out - T) ** 2)) < 1e-13
    idx = np.concatenate([rng.choice(16384, 6, replace=False),              # W1
                          16384 + rng.choice(256, 3, replace=False),       # b1
                          16640 + rng.choice(65536, 6, replace=False),     # W2
                          82176 + rng.choice(256, 3, replace=False),       # b2
                          82432 + rng.choice(768, 4, replace=False),       # W3
                          83200 + np.arange(3)])                           # b3
    h = 1e-6
    for i in idx:
        Wp, Wm = W.copy(), W.copy()
        Wp[i] += h
        Wm[i] -= h
        fd = (orc.mlp_loss_grad(Wp, S, T)[0] - orc.mlp_loss_grad(Wm, S, T)[0]) / (2 * h)
        assert abs(g[i] - fd) < 1e-7 * max(1.0, abs(fd))


# --------------------------------------------------------------------------- Matern kernels

MATERN = {"matern12": 0.5, "matern32": 1.5, "matern52": 2.5}


def _matern_bessel(r, l, nu, p):
    """Matern kernel from its general definition with the modified Bessel function
    (Rasmussen & Williams Eq. 4.14), independent of the half-integer closed forms."""
    from scipy.special import gamma, kv
    z = np.sqrt(2.0 * p) * np.asarray(r, dtype=np.float64) / l
    out = np.full(z.shape, nu)
    nz = z > 0
    out[nz] = nu * 2.0 ** (1.0 - p) / gamma(p) * z[nz] ** p * kv(p, z[nz])
    return out


@pytest.mark.parametrize("kernel", sorted(MATERN))
def test_matern_against_bessel_definition(orc, kernel):
    A = dg.random_points(7, 4, seed=11)
    B = dg.random_points(9, 4, seed=12)
    l, nu = 0.7, 1.3
    K = orc.kernel_cross(A, B, l, nu, kernel)
    r = cdist(A, B)
    assert max_rel(K, _matern_bessel(r, l, nu, MATERN[kernel])) < 1e-12
    assert np.allclose(np.diag(orc.kernel_cross(A, A, l, nu, kernel)), nu, rtol=0, atol=0)


def test_matern12_is_markov_in_one_dimension(orc):
    """The order-1/2 Matern kernel in one dimension is the Ornstein-Uhlenbeck
    covariance: for sorted inputs and no noise its inverse is tridiagonal."""
    x = np.sort(dg.uniform(21, 0, 40, 0.0, 6.0)).reshape(-1, 1)
    K = orc.cov_train(x, (0.8, 1.1, 0.0), kernel="matern12")
    Kinv = orc.chol_inverse(orc.cholesky(K))
    off = np.abs(np.triu(Kinv, 2))
    assert off.max() < 1e-9 * np.abs(Kinv).max()
    assert np.abs(np.diag(Kinv, 1)).min() > 1e-3 * np.abs(Kinv).max()


@pytest.mark.parametrize("kernel", sorted(MATERN))
def test_matern_n2_closed_forms_and_gradient(orc, kernel):
    l, nu, s2 = 1.3, 0.9, 0.2
    X = np.array([[0.0, 0.5], [0.75, -0.25]])
    y = np.array([0.4, -1.1])
    xs = np.array([[0.25, 0.25]])
    r = np.sqrt(2 * 0.75 ** 2)
    a, c = nu + s2, _matern_bessel([r], l, nu, MATERN[kernel])[0]
    det = a * a - c * c
    Kinv = np.array([[a, -c], [-c, a]]) / det
    alpha = Kinv @ y
    kh = _matern_bessel(np.sqrt([2 * 0.25 ** 2, 2 * 0.5 ** 2]), l, nu, MATERN[kernel])
    mu, va, _ = orc.predict(X, y, xs, (l, nu, s2), kernel=kernel)
    assert abs(mu[0] - kh @ alpha) < 1e-13
    assert abs(va[0] - (nu - kh @ Kinv @ kh)) < 1e-13
    f = orc.nlml(X, y, (l, nu, s2), kernel=kernel)
    assert abs(f - (0.5 * y @ alpha + 0.5 * np.log(det) + np.log(2 * np.pi))) < 1e-13
    # the length-scale derivative of c by a central difference of the Bessel form
    h = 1e-6
    dc = (_matern_bessel([r], l * np.exp(h), nu, MATERN[kernel])[0]
          - _matern_bessel([r], l * np.exp(-h), nu, MATERN[kernel])[0]) / (2 * h)
    W = Kinv - np.outer(alpha, alpha)
    g_expect = [0.5 * 2 * W[0, 1] * dc, 0.5 * (W[0, 0] * nu + W[1, 1] * nu + 2 * W[0, 1] * c),
                0.5 * s2 * (W[0, 0] + W[1, 1])]
    _, g = orc.nlml_grad(X, y, (l, nu, s2), kernel=kernel)
    assert max_rel(g, g_expect) < 1e-8


@pytest.mark.parametrize("kernel", sorted(MATERN))
def test_matern_gradient_against_central_differences(orc, kernel):
    X, y, _, _ = small_set(n=40, d=4, seed=1014)
    hyp = (0.8, 1.2, 0.07)
    f, g = orc.nlml_grad(X, y, hyp, kernel=kernel)
    assert abs(f - orc.nlml(X, y, hyp, kernel=kernel)) == 0.0
    h = 1e-5
    th = np.log(hyp)
    fd = np.empty(3)
    for p in range(3):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (orc.nlml(X, y, np.exp(tp), kernel=kernel) - orc.nlml(X, y, np.exp(tm), kernel=kernel)) / (2 * h)
    assert max_rel(g, fd, floor=1e-8 * np.linalg.norm(fd)) < 1e-7


@pytest.mark.parametrize("kernel", sorted(MATERN))
def test_matern_long_length_scale_limit(orc, kernel):
    X = dg.random_points(30, 3, seed=8)
    Xs = dg.random_points(5, 3, seed=9)
    y = dg.uniform(10, 0, 30, -1, 1)
    nu, s2, n = 0.8, 0.25, 30
    one = np.ones(n)
    alpha = (y - nu * one * (one @ y) / (s2 + n * nu)) / s2
    mu, va, _ = orc.predict(X, y, Xs, (1e9, nu, s2), kernel=kernel)
    assert max_rel(mu, np.full(5, nu * one @ alpha), 1e-3) < 1e-6
    assert np.all(np.abs(va - (nu - nu * nu * n / (s2 + n * nu))) < 1e-6)
