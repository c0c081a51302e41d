"""FP64 CUDA path against the FP64 CPU oracle, element by element, through the C ABI.

Tolerance: 1e-9 relative (norm-wise, and worst element against a floor of
1e-12 nu for mean/variance) on mean, variance, covariance and NLML; 1e-9 on
the factor; the gradient to 1e-9 of the oracle and 1e-6 of central finite
differences.  Sizes span several tiles and a ragged tail.
"""
import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import rel, max_rel

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat
    return gprat


def check_predict(g, orc, X, y, Xs, hyp, n_tiles, noisy=False, cov=True):
    with g.GP(X, y, hyp, n_tiles=n_tiles, noisy_test_var=noisy) as gp:
        mu_o, va_o, cv_o = orc.predict(X, y, Xs, hyp, noisy=noisy, cov=cov)
        mu, va = gp.predict_var(Xs)
        assert rel(mu, mu_o) < TOL, rel(mu, mu_o)
        assert max_rel(mu, mu_o, 1e-12 * hyp[1] + 1e-3 * np.abs(mu_o).max()) < TOL
        assert rel(va, va_o) < TOL, rel(va, va_o)
        assert max_rel(va, va_o, 1e-12 * hyp[1]) < 10 * TOL
        assert rel(gp.predict_mean(Xs), mu_o) < TOL
        if cov:
            mu2, cv = gp.predict_full_cov(Xs)
            assert rel(cv, cv_o) < TOL, rel(cv, cv_o)
            assert np.array_equal(cv, cv.T)
            assert rel(np.diag(cv), va) < TOL
            assert rel(mu2, mu_o) < TOL
        f = gp.nlml()
        f_o = orc.nlml(X, y, hyp)
        assert abs(f - f_o) < TOL * abs(f_o), (f, f_o)


def test_config1_mean_variance_nlml(g, orc):
    """N = M = 1024, 8 lagged regressors, 4 x 4 tiles of 256, (l, nu, sigma^2) = (1, 1, 0.1)."""
    X, y, Xs, _ = dg.msd_dataset(1024, 1024, 8, seed=1001)
    check_predict(g, orc, X, y, Xs, (1.0, 1.0, 0.1), n_tiles=4)


@pytest.mark.parametrize("n,m,d,n_tiles", [(1000, 77, 3, 4), (130, 5, 2, 3), (1, 1, 1, 1),
                                           (65, 64, 8, 2), (700, 200, 8, 16)])
def test_ragged_sizes(g, orc, n, m, d, n_tiles):
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed=900 + n)
    check_predict(g, orc, X, y, Xs, (0.9, 1.2, 0.07), n_tiles=n_tiles, noisy=(n % 2 == 0))


def test_many_regressors_nondegenerate(g, orc):
    X, y, Xs, _ = dg.msd_dataset(512, 128, 128, seed=1002)
    check_predict(g, orc, X, y, Xs, (np.sqrt(128.0), 1.0, 0.1), n_tiles=4, cov=False)


def test_many_regressors_degenerate_unit_lengthscale(g, orc):
    X, y, Xs, _ = dg.msd_dataset(256, 64, 128, seed=1003)
    check_predict(g, orc, X, y, Xs, (1.0, 1.0, 0.1), n_tiles=2, cov=False)


def test_automatic_tile_count(g, orc):
    """n_tiles = 0 takes gp_auto_tiles(n): 1000 points -> 4 tiles of 256 (ragged
    last tile), same results as the oracle."""
    X, y, Xs, _ = dg.msd_dataset(1000, 96, 8, seed=1005)
    assert g.auto_tiles(1000) == 4
    with g.GP(X, y, (1.0, 1.0, 0.1), n_tiles=0) as gp:
        info = gp.info()
        assert info["n_tiles"] == 4 and info["tile"] == 256
    check_predict(g, orc, X, y, Xs, (1.0, 1.0, 0.1), n_tiles=0, cov=False)


def test_tile_count_invariance_and_factor(g, orc):
    X, y, Xs, _ = dg.msd_dataset(1024, 128, 8, seed=1001)
    hyp = (1.0, 1.0, 0.1)
    K = orc.cov_train(X, hyp)
    L_o = orc.cholesky(K)
    outs = []
    for T in (1, 4, 16):
        with g.GP(X, y, hyp, n_tiles=T) as gp:
            L = gp.get_factor()
            assert rel(L, L_o) < TOL
            assert np.all(np.triu(L, 1) == 0)
            assert np.linalg.norm(L @ L.T - K) / np.linalg.norm(K) < 1e-13
            outs.append(gp.predict_var(Xs))
    for mu, va in outs[1:]:
        assert rel(mu, outs[0][0]) < 1e-11 and rel(va, outs[0][1]) < 1e-11


def test_gradient_against_oracle_and_finite_differences(g, orc):
    X, y, _, _ = dg.msd_dataset(600, 0, 8, seed=1004)
    hyp = (0.8, 1.3, 0.05)
    f_o, g_o = orc.nlml_grad(X, y, hyp)
    with g.GP(X, y, hyp, n_tiles=5) as gp:
        f, gr = gp.nlml_grad()
        assert abs(f - f_o) < TOL * abs(f_o)
        assert max_rel(gr, g_o, 1e-8 * np.linalg.norm(g_o)) < TOL
        h = 1e-5
        th = np.log(hyp)
        fd = np.empty(3)
        for p in range(3):
            vals = []
            for s in (+1, -1):
                t = th.copy()
                t[p] += s * h
                gp.set_hyper(np.exp(t))
                vals.append(gp.nlml())
            fd[p] = (vals[0] - vals[1]) / (2 * h)
        assert max_rel(gr, fd, 1e-8 * np.linalg.norm(fd)) < 1e-6


def test_adam_trajectory_matches_oracle(g, orc):
    X, y, _, _ = dg.msd_dataset(300, 0, 8, seed=1005)
    hyp = (1.0, 1.0, 0.1)
    h_o, hist_o = orc.optimize(X, y, hyp, steps=12, lr=0.1, trainable=(1, 0, 1))
    with g.GP(X, y, hyp, trainable=(1, 0, 1), n_tiles=3) as gp:
        hist = gp.optimize(12, lr=0.1)
        (l, nu, s2), _ = gp.get_hyper()
        assert max_rel(hist, hist_o) < 1e-9
        assert max_rel([l, nu, s2], h_o) < 1e-9
        assert nu == 1.0
        st = gp.get_state()
        assert st["adam_t"] == 12
        # checkpoint / resume: continuing from a restored state equals an uninterrupted run
        more = gp.optimize(3, lr=0.1)
        gp.set_state(st)
        again = gp.optimize(3, lr=0.1)
        assert max_rel(more, again) < 1e-12


def test_not_positive_definite_reports_pivot(g):
    X = np.zeros((200, 3))
    y = np.ones(200)
    with pytest.raises(g.GPError) as e:
        with g.GP(X, y, (1.0, 1.0, 0.0), n_tiles=2) as gp:
            gp.factor()
    assert e.value.status == g.GP_ERR_NOT_PD and e.value.info == 1


def test_jitter_retry_recovers_from_a_singular_matrix(g):
    """Identical inputs with sigma^2 = 0 give K = nu 11^T, singular.  With
    jitter retries the first try (sigma^2 = 1e-10 nu) factors, the added
    jitter is reported and kept in the hyperparameters, and the mean at the
    training input is n nu / (n nu + sigma^2) = 1 - 5e-13 for y = 1."""
    X = np.zeros((200, 3))
    y = np.ones(200)
    with g.GP(X, y, (1.0, 1.0, 0.0), n_tiles=2, jitter_retries=3) as gp:
        gp.factor()
        info = gp.info()
        assert info["jitter_added"] == pytest.approx(1e-10, rel=1e-12)
        (l, nu, s2), _ = gp.get_hyper()
        assert s2 == pytest.approx(1e-10, rel=1e-12) and (l, nu) == (1.0, 1.0)
        mu = gp.predict_mean(X[:4])
        assert np.allclose(mu, 200.0 / (200.0 + 1e-10), rtol=1e-4)
    # retries off (the default): the same matrix is refused, sigma^2 untouched
    with g.GP(X, y, (1.0, 1.0, 0.0), n_tiles=2) as gp:
        with pytest.raises(g.GPError) as e:
            gp.factor()
        assert e.value.status == g.GP_ERR_NOT_PD
        assert gp.get_hyper()[0][2] == 0.0 and gp.info()["jitter_added"] == 0.0


def test_device_buffers_match_host_buffers(g, orc):
    import torch
    X, y, Xs, _ = dg.msd_dataset(400, 100, 8, seed=1006)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=4) as gp:
        mu_h, va_h = gp.predict_var(Xs)
    Xd, yd, Xsd = (torch.from_numpy(a).cuda() for a in (X, y, Xs))
    with g.GP(Xd, yd, hyp, n_tiles=4) as gp:
        mu_d, va_d = gp.predict_var(Xsd)
        assert mu_d.is_cuda
        _, cv_d = gp.predict_full_cov(Xsd)
        torch.cuda.synchronize()
    assert np.array_equal(mu_d.cpu().numpy(), mu_h) and np.array_equal(va_d.cpu().numpy(), va_h)
    assert rel(np.diag(cv_d.cpu().numpy()), va_h) < TOL


def test_oracle_parity_several_tiles_ragged_test_set(g, orc):
    """N = 4096 over 16 tiles of 256, M = 70 (ragged), full covariance."""
    X, y, Xs, _ = dg.msd_dataset(4096, 70, 8, seed=1001)
    check_predict(g, orc, X, y, Xs, (1.0, 1.0, 0.1), n_tiles=16)


def test_full_size_properties(g, orc):
    """N = 32768, M = 8192, 8 regressors, 128 tiles of 256 (the benchmark's
    launch configuration).  The oracle cannot factor this size in test time, so
    the outputs are checked against CPU arithmetic on sampled rows:
    (K alpha)_i = y_i, mean_j = k*_j^T alpha, and 0 <= var <= nu."""
    n, m = 32768, 8192
    X, y, Xs, _ = dg.msd_dataset(n, m, 8, seed=1002)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=128) as gp:
        mu, va = gp.predict_var(Xs)
        alpha = gp.get_alpha()
        f = gp.nlml()
    rows = np.linspace(0, n - 1, 40).astype(int)
    Kr = orc.se_cross(X[rows], X, hyp[0], hyp[1])
    resid = Kr @ alpha + hyp[2] * alpha[rows] - y[rows]
    assert np.linalg.norm(resid) / np.linalg.norm(y[rows]) < 1e-9
    cols = np.linspace(0, m - 1, 40).astype(int)
    Kc = orc.se_cross(Xs[cols], X, hyp[0], hyp[1])
    assert rel(mu[cols], Kc @ alpha) < 1e-10
    assert np.all(va >= 0.0) and np.all(va <= hyp[1])
    assert np.isfinite(f) and f < 0.5 * n * np.log(2 * np.pi * (hyp[1] + hyp[2])) + y @ y
