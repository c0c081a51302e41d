"""GP_FP64_OZAKI: the FP64 path with its O(n^3) and O(n^2 m) products (the
factorisation's trailing updates, the V solve's updates, the triangular
inverse's accumulations, K^{-1} = L^{-T} L^{-1} and the full covariance) as
exact digit products on the BF16 tensor cores, against the FP64 oracle at the
FP64 path's tolerance (1e-9 relative on mean, variance, covariance, NLML,
gradient and factor) and against the native FP64 GPU path.
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


@pytest.mark.parametrize("n,m,d,n_tiles,ls", [(1024, 300, 8, 4, 1.0), (1000, 77, 3, 4, 0.7), (777, 64, 5, 3, 1.3),
                                              (2048, 128, 128, 8, 128 ** 0.5), (256, 10, 8, 1, 1.0)])
def test_fp64_ozaki_against_oracle(g, orc, n, m, d, n_tiles, ls):
    """Tiles of 256 with several steps, a ragged n (identity padding), tiles of
    384 (three 128-row blocks per tile edge), 128 regressors, one tile."""
    X, y, Xs, _ = dg.msd_dataset(n, m, d, seed=1041 + n + d)
    hyp = (ls, 1.0, 0.1)
    mu_o, va_o, cv_o = orc.predict(X, y, Xs, hyp, cov=True)
    f_o, g_o = orc.nlml_grad(X, y, hyp)
    K = orc.cov_train(X, hyp)
    L_o = orc.cholesky(K)
    with g.GP(X, y, hyp, n_tiles=n_tiles, precision="fp64_ozaki") as gp:
        mu, va, cv = gp.predict(Xs, mean=True, var=True, cov=True)
        f, gr = gp.nlml_grad()
        L = gp.get_factor()
        info = gp.info()
    errs = {"mean": rel(mu, mu_o), "mean_worst": max_rel(mu, mu_o, 1e-3 * np.abs(mu_o).max()),
            "var": rel(va, va_o), "var_worst": max_rel(va, va_o, 1e-12), "nlml": abs(f - f_o) / abs(f_o),
            "grad": rel(gr, g_o), "factor": rel(L, L_o), "cov": rel(cv, cv_o), "tile": info["tile"]}
    print("fp64_ozaki vs oracle", n, m, d, errs)
    assert info["tile"] % 128 == 0
    assert np.array_equal(cv, cv.T)
    for k in ("mean", "var", "nlml", "grad", "factor", "cov"):
        assert errs[k] < TOL, (k, errs[k])
    assert errs["mean_worst"] < 10 * TOL and errs["var_worst"] < 10 * TOL


def test_fp64_ozaki_matches_native_fp64_path(g):
    """N = 8192, 32 tiles of 256: the emulated factor against the native FP64
    GPU factor, and the outputs built on it."""
    X, y, Xs, _ = dg.msd_dataset(8192, 512, 8, seed=1002)
    hyp = (1.0, 1.0, 0.1)
    out = {}
    for prec in ("fp64", "fp64_ozaki"):
        with g.GP(X, y, hyp, n_tiles=32, precision=prec) as gp:
            mu, va, cv = gp.predict(Xs, mean=True, var=True, cov=True)
            f, gr = gp.nlml_grad()
            out[prec] = (mu, va, f, gr, gp.get_alpha(), cv)
    a, b = out["fp64_ozaki"], out["fp64"]
    errs = {"mean": rel(a[0], b[0]), "var": rel(a[1], b[1]), "nlml": abs(a[2] - b[2]) / abs(b[2]),
            "grad": rel(a[3], b[3]), "alpha": rel(a[4], b[4]), "cov": rel(a[5], b[5])}
    print("fp64_ozaki vs fp64 @8192", errs)
    for k, v in errs.items():
        assert v < TOL, (k, v)


def test_fp64_ozaki_not_pd_reports_pivot(g):
    X = np.zeros((300, 3))
    with pytest.raises(g.GPError) as e:
        with g.GP(X, np.ones(300), (1.0, 1.0, 0.0), n_tiles=3, precision="fp64_ozaki") as gp:
            gp.factor()
    assert e.value.status == g.GP_ERR_NOT_PD and e.value.info == 1
