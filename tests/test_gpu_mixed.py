"""Mixed-precision path (FP32 diagonal-tile factor, split-BF16 tensor-core
products, FP64-residual refinement, exactly corrected variances) against the
FP64 oracle and against the FP64 GPU path.

alpha and the predictive mean are refined to FP64 accuracy (mean = K_{Z*,Z}
alpha) and the variances corrected to FP64 level: both to 1e-8 relative,
norm-wise and element by element.  The factor itself, the NLML (through
log|K|), the gradient and the full covariance are FP32-accurate: their bounds
below follow from FP32 unit roundoff (6e-8) times the growth measured at
these sizes, with a margin of 10 or more.  Reported errors are printed for the
record (pytest -s).
"""
import time

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2505_00136_gb300 import datagen as dg
from _util import rel, max_rel

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-8
VAR_TOL = 1e-8
# The NLML takes log|K| from the FP32-accurate factor: the FP32 errors of the
# trailing updates reach every pivot, and log|K| sums them over all n pivots
# (it grows with n and with kappa(K)).  Measured relative NLML errors:
# 2e-6 (n = 512), 4.5e-5 (n = 4096, 8 regressors), 1.2e-4 (n = 2048, 128
# regressors with l = sqrt(128): kappa(K) = 1.5e4 against 5e3), 4.8e-4
# (n = 32768).  The bound covers n <= 4096 with a margin of four.
NLML_TOL = 5e-4


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat
    return gprat


@pytest.mark.parametrize("n,m,d,n_tiles", [(1024, 1024, 8, 4), (1000, 77, 3, 4), (130, 5, 2, 1),
                                           (2048, 200, 8, 16),
                                           (1500, 150, 8, 6), (1200, 64, 5, 5)])   # short last super-block of the solves
def test_mixed_against_oracle(g, orc, n, m, d, n_tiles):
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed=1001 + n)
    hyp = (1.0, 1.0, 0.1)
    mu_o, va_o, _ = orc.predict(X, y, Xs, hyp)
    f_o = orc.nlml(X, y, hyp)
    K = orc.cov_train(X, hyp)
    alpha_o = sla.cho_solve(sla.cho_factor(K, lower=True), y)
    with g.GP(X, y, hyp, n_tiles=n_tiles, precision="mixed") as gp:
        mu, va = gp.predict_var(Xs)
        alpha = gp.get_alpha()
        f = gp.nlml()
        info = gp.info()
        L = gp.get_factor()
    errs = {"alpha": rel(alpha, alpha_o), "mean": rel(mu, mu_o), "var": rel(va, va_o),
            "nlml": abs(f - f_o) / abs(f_o), "factor": rel(L, orc.cholesky(K)),
            "refine_iters": info["refine_iters"], "refine_residual": info["refine_residual"]}
    print("mixed vs oracle", n, m, d, errs)
    assert info["tile"] % 128 == 0
    assert errs["alpha"] < 1e-10
    assert errs["mean"] < MEAN_TOL
    assert errs["var"] < VAR_TOL
    # FP32-accurate factor: its own error, and the NLML through log|K|, stay at that level
    assert errs["factor"] < 1e-4
    assert errs["nlml"] < NLML_TOL


@pytest.mark.parametrize("n,m,d,n_tiles,ls", [(4096, 512, 8, 16, 1.0), (4000, 300, 8, 16, 1.0),
                                              (2048, 256, 128, 8, 128 ** 0.5)])
def test_mixed_tiles_of_256_against_oracle(g, orc, n, m, d, n_tiles, ls):
    """The bench's tiling (tiles of 256: 128 x 256 tensor units, super-panels of
    four tile columns with multi-segment trailing updates, multi-segment W
    sweeps, the inverse in blocks of four) against the oracle, element-wise:
    16 tiles (four super-panels), a ragged n = 4000 (padded to 4096 with an
    identity block), and 128 regressors with l = sqrt(128)."""
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed=1021 + n + d)
    hyp = (ls, 1.0, 0.1)
    mu_o, va_o, _ = orc.predict(X, y, Xs, hyp)
    with_grad = n <= 2048   # the oracle's unblocked K^{-1} costs n^3: gradient at the smaller size only
    f_o, g_o = orc.nlml_grad(X, y, hyp) if with_grad else (orc.nlml(X, y, hyp), None)
    with g.GP(X, y, hyp, n_tiles=n_tiles, precision="mixed") as gp:
        mu, va = gp.predict_var(Xs)
        f, gr = gp.nlml_grad()
        info = gp.info()
    errs = {"mean": rel(mu, mu_o), "mean_worst": max_rel(mu, mu_o, 1e-3 * np.abs(mu_o).max()),
            "var": rel(va, va_o), "var_worst": max_rel(va, va_o, 1e-12),
            "nlml": abs(f - f_o) / abs(f_o), "tile": info["tile"],
            "n_tiles": info["n_tiles"], "refine_iters": info["refine_iters"]}
    if with_grad:
        errs["grad"] = rel(gr, g_o)
    print("mixed tiles of 256 vs oracle", n, m, d, errs)
    assert info["tile"] == 256 and info["n_tiles"] == n_tiles
    assert errs["mean"] < MEAN_TOL and errs["mean_worst"] < MEAN_TOL
    assert errs["var"] < VAR_TOL and errs["var_worst"] < VAR_TOL
    assert errs["nlml"] < NLML_TOL
    if with_grad:
        assert errs["grad"] < 1e-3


@pytest.mark.parametrize("n,m,d,n_tiles,ls,noisy", [(1000, 200, 40, 4, 4.0, False), (777, 130, 160, 3, 8.0, True),
                                                    (2048, 256, 128, 8, 1.0, False)])
def test_mixed_tensor_core_distances_against_oracle(g, orc, n, m, d, n_tiles, ls, noisy):
    """From 32 regressors up the mixed path forms every squared distance as
    |z_i|^2 + |z_j|^2 - 2 z_i . z_j with the inner products an exact digit
    product on the tensor cores (K tiles, K_{Z*,Z}, K_{Z*,Z*}).  Padded
    regressor counts (40 -> 64), two exact chunks along the regressors (160),
    tiles of 384 (three 128-row blocks per tile edge), ragged n and m, the
    noisy test prior and the degenerate l = 1 at 128 regressors."""
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed=1031 + n + d)
    hyp = (ls, 1.0, 0.1)
    mu_o, va_o, cv_o = orc.predict(X, y, Xs, hyp, cov=True, noisy=noisy)
    with g.GP(X, y, hyp, n_tiles=n_tiles, precision="mixed", noisy_test_var=noisy) as gp:
        mu, va, cv = gp.predict(Xs, mean=True, var=True, cov=True)
        alpha = gp.get_alpha()
    K = orc.cov_train(X, hyp)
    alpha_o = sla.cho_solve(sla.cho_factor(K, lower=True), y)
    errs = {"alpha": rel(alpha, alpha_o), "mean": rel(mu, mu_o),
            "mean_worst": max_rel(mu, mu_o, 1e-3 * np.abs(mu_o).max() + 1e-300),
            "var": rel(va, va_o), "var_worst": max_rel(va, va_o, 1e-12), "cov": rel(cv, cv_o)}
    print("mixed tensor-core distances vs oracle", n, m, d, errs)
    assert errs["alpha"] < 1e-10
    assert errs["mean"] < MEAN_TOL and errs["mean_worst"] < MEAN_TOL
    assert errs["var"] < VAR_TOL and errs["var_worst"] < VAR_TOL
    # K_{Z*,Z*} - W^T W with the FP32-accurate W: FP32 level, amplified where the
    # posterior covariance is small against the prior
    assert errs["cov"] < 1e-3
    assert np.array_equal(cv, cv.T)
    # test points far from every training point: K_{Z*,Z} underflows to ~0, so the
    # covariance is the tensor-core prior K_{Z*,Z*} itself, checked at FP64 level
    Xf = Xs + 10.0 * ls
    _, _, cf_o = orc.predict(X, y, Xf, hyp, cov=True, noisy=noisy)
    with g.GP(X, y, hyp, n_tiles=n_tiles, precision="mixed", noisy_test_var=noisy) as gp:
        _, _, cf = gp.predict(Xf, mean=True, var=False, cov=True)
    print("prior", rel(cf, cf_o), max_rel(cf, cf_o, 1e-300))
    assert rel(cf, cf_o) < 1e-12


def test_mixed_not_pd(g):
    X = np.zeros((300, 3))
    with pytest.raises(g.GPError) as e:
        with g.GP(X, np.ones(300), (1.0, 1.0, 0.0), n_tiles=2, precision="mixed") as gp:
            gp.factor()
    assert e.value.status == g.GP_ERR_NOT_PD and e.value.info == 1


def test_mixed_vs_fp64_full_size(g):
    """N = 32768, M = 8192, D = 8: the mixed path against the FP64 GPU path."""
    import time
    X, y, Xs, _ = dg.msd_dataset(32768, 8192, 8, seed=1002)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=128, precision="mixed") as gp:   # the bench's tiling: tiles of 256
        t0 = time.perf_counter()
        mu_m, va_m = gp.predict_var(Xs)
        t_mixed = time.perf_counter() - t0
        f_m = gp.nlml()
        info = gp.info()
    with g.GP(X, y, hyp, n_tiles=128) as gp:
        t0 = time.perf_counter()
        mu_d, va_d = gp.predict_var(Xs)
        t_fp64 = time.perf_counter() - t0
        f_d = gp.nlml()
    errs = {"mean": rel(mu_m, mu_d), "var": rel(va_m, va_d), "nlml": abs(f_m - f_d) / abs(f_d),
            "refine_iters": info["refine_iters"], "refine_residual": info["refine_residual"],
            "t_mixed_s": t_mixed, "t_fp64_s": t_fp64}
    errs["mean_worst"] = max_rel(mu_m, mu_d, 1e-3 * np.abs(mu_d).max())
    errs["var_worst"] = max_rel(va_m, va_d, 1e-12)
    print("mixed vs fp64 @32768", errs)
    assert errs["mean"] < MEAN_TOL and errs["mean_worst"] < MEAN_TOL
    assert errs["var"] < VAR_TOL and errs["var_worst"] < VAR_TOL
    assert t_mixed < t_fp64 / 2


def test_mixed_gradient_full_cov_and_optimize(g, orc):
    X, y, Xs, _ = dg.msd_dataset(1024, 256, 8, seed=1004)
    hyp = (0.9, 1.1, 0.08)
    f_o, g_o = orc.nlml_grad(X, y, hyp)
    mu_o, va_o, cv_o = orc.predict(X, y, Xs, hyp, cov=True)
    h_o, hist_o = orc.optimize(X, y, hyp, steps=5, lr=0.1)
    with g.GP(X, y, hyp, n_tiles=4, precision="mixed") as gp:
        f, gr = gp.nlml_grad()
        mu, cv = gp.predict_full_cov(Xs)
        hist = gp.optimize(5, lr=0.1)
    errs = {"grad": rel(gr, g_o), "nlml": abs(f - f_o) / abs(f_o), "cov": rel(cv, cv_o),
            "mean": rel(mu, mu_o), "hist": rel(hist, hist_o)}
    print("mixed gradient/cov", errs)
    assert errs["mean"] < MEAN_TOL
    assert errs["grad"] < 1e-3
    assert errs["cov"] < 1e-4
    assert np.array_equal(cv, cv.T)
    assert errs["hist"] < 1e-4
    assert hist[-1] < hist[0]


def test_uncorrected_variance_is_fp32_level(g, orc):
    X, y, Xs, _ = dg.msd_dataset(1024, 300, 8, seed=1011)
    hyp = (1.0, 1.0, 0.1)
    _, va_o, _ = orc.predict(X, y, Xs, hyp)
    with g.GP(X, y, hyp, n_tiles=8, precision="mixed", var_correction=False) as gp:
        _, va_u = gp.predict_var(Xs)
    with g.GP(X, y, hyp, n_tiles=8, precision="mixed") as gp:
        _, va_c = gp.predict_var(Xs)
        _, va_c2 = gp.predict_var(Xs)      # second call reuses the cached K digits
    e_u, e_c = rel(va_u, va_o), rel(va_c, va_o)
    print("variance uncorrected / corrected", e_u, e_c)
    assert 1e-9 < e_u < 1e-3
    assert e_c < VAR_TOL and rel(va_c2, va_c) < 1e-14


def test_solve_barrier_wait_expires_and_device_stays_usable(g):
    """A bounded wait of the persistent FP32 solve runs out: the last CTA never
    arrives at the first grid barrier (host-set test aid, 20 ms bound), the
    factorising call returns GP_ERR_TIMEOUT, and the same handle and context
    then give the unstalled result bit for bit."""
    X, y, Xs, _ = dg.msd_dataset(1024, 64, 8, seed=91)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=4, precision="mixed") as ref:
        mu_r, va_r = ref.predict_var(Xs)
    with g.GP(X, y, hyp, n_tiles=4, precision="mixed") as gp:
        gp.solve_stall(True, 20000)
        t0 = time.perf_counter()
        with pytest.raises(g.GPError) as e:
            gp.predict_var(Xs)
        assert e.value.status == g.GP_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 20.0
        gp.solve_stall(False)
        mu, va = gp.predict_var(Xs)
    assert np.array_equal(mu, mu_r) and np.array_equal(va, va_r)
