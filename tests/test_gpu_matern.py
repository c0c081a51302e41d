"""Matern kernels (order 1/2, 3/2, 5/2; the paper's future work) on every
path against the oracle: FP64 and the emulated FP64 path at 1e-9 on mean,
variance, covariance, NLML and gradient; the mixed path at 1e-8 on mean and
variance (with direct-difference and tensor-core distances) and at its
FP32-factor level on the NLML and gradient.
"""
import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import rel, max_rel

pytestmark = pytest.mark.gpu

KERNELS = ["matern12", "matern32", "matern52"]


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat
    return gprat


def oracle_outputs(orc, X, y, Xs, hyp, kernel):
    mu, va, cv = orc.predict(X, y, Xs, hyp, cov=True, kernel=kernel)
    f, gr = orc.nlml_grad(X, y, hyp, kernel=kernel)
    return mu, va, cv, f, gr


@pytest.mark.parametrize("precision", ["fp64", "fp64_ozaki"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_matern_fp64_paths_against_oracle(g, orc, kernel, precision):
    X, y, Xs, _ = dg.msd_dataset(1000, 90, 5, seed=1051)
    hyp = (1.4, 0.9, 0.08)
    mu_o, va_o, cv_o, f_o, g_o = oracle_outputs(orc, X, y, Xs, hyp, kernel)
    with g.GP(X, y, hyp, n_tiles=4, precision=precision, kernel=kernel) as gp:
        mu, va, cv = gp.predict(Xs, mean=True, var=True, cov=True)
        f, gr = gp.nlml_grad()
    errs = {"mean": rel(mu, mu_o), "var": rel(va, va_o), "cov": rel(cv, cv_o),
            "nlml": abs(f - f_o) / abs(f_o), "grad": rel(gr, g_o)}
    print(precision, kernel, errs)
    for k, v in errs.items():
        assert v < 1e-9, (k, v)
    assert max_rel(va, va_o, 1e-12) < 1e-8


@pytest.mark.parametrize("d", [8, 40])
@pytest.mark.parametrize("kernel", KERNELS)
def test_matern_mixed_against_oracle(g, orc, kernel, d):
    X, y, Xs, _ = dg.msd_dataset(1024, 150, d, seed=1053 + d)
    hyp = (1.2 * (d / 8) ** 0.5, 1.1, 0.1)
    mu_o, va_o, _, f_o, g_o = oracle_outputs(orc, X, y, Xs, hyp, kernel)
    with g.GP(X, y, hyp, n_tiles=4, precision="mixed", kernel=kernel) as gp:
        mu, va = gp.predict_var(Xs)
        f, gr = gp.nlml_grad()
    errs = {"mean": rel(mu, mu_o), "mean_worst": max_rel(mu, mu_o, 1e-3 * np.abs(mu_o).max()),
            "var": rel(va, va_o), "var_worst": max_rel(va, va_o, 1e-12),
            "nlml": abs(f - f_o) / abs(f_o), "grad": rel(gr, g_o)}
    print("mixed", kernel, d, errs)
    assert errs["mean"] < 1e-8 and errs["mean_worst"] < 1e-8
    assert errs["var"] < 1e-8 and errs["var_worst"] < 1e-8
    assert errs["nlml"] < 5e-4 and errs["grad"] < 1e-2
