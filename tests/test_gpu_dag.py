"""Persistent tile-DAG scheduler (one launch walking the Cholesky task graph).

Per tile it applies the same operations in the same order as the stream
scheduler, so the factor must be bitwise identical; pivot failures and the
bounded dependency waits must come back as status codes with the device
still usable.
"""
import time

import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat
    return gprat


@pytest.mark.parametrize("n,n_tiles", [(2048, 8), (1000, 4), (4096, 16), (130, 3), (64, 1)])
def test_persistent_factor_bitwise_equals_stream(g, orc, n, n_tiles):
    X, y, Xs, _ = dg.msd_dataset(n, 50, 8, seed=500 + n)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=n_tiles) as a:
        La = a.get_factor()
        fa = a.nlml()
        mu_a, va_a = a.predict_var(Xs)
    with g.GP(X, y, hyp, n_tiles=n_tiles, scheduler="persistent") as p:
        Lp = p.get_factor()
        fp = p.nlml()
        mu_p, va_p = p.predict_var(Xs)
    assert np.array_equal(La, Lp)
    assert fa == fp
    assert np.array_equal(mu_a, mu_p) and np.array_equal(va_a, va_p)
    mu_o, va_o, _ = orc.predict(X, y, Xs, hyp)
    assert rel(mu_p, mu_o) < 1e-9 and rel(va_p, va_o) < 1e-9


def test_persistent_reports_pivot_failure(g):
    X = np.zeros((600, 3))
    with pytest.raises(g.GPError) as e:
        with g.GP(X, np.ones(600), (1.0, 1.0, 0.0), n_tiles=4, scheduler="persistent") as gp:
            gp.factor()
    assert e.value.status == g.GP_ERR_NOT_PD and e.value.info == 1


def test_bounded_wait_times_out_and_device_stays_usable(g):
    X, y, _, _ = dg.msd_dataset(1024, 0, 8, seed=77)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=4, scheduler="persistent", dag_timeout_ms=300) as gp:
        gp.dag_stall_tile(2, 1)            # a dependency counter that nothing completes
        t0 = time.perf_counter()
        with pytest.raises(g.GPError) as e:
            gp.factor()
        assert e.value.status == g.GP_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        gp.dag_stall_tile(-1)
        gp.factor()                        # same handle, same context: works again
        L = gp.get_factor()
    with g.GP(X, y, hyp, n_tiles=4) as ref:
        assert np.array_equal(L, ref.get_factor())


def test_persistent_optimize_matches_stream(g):
    X, y, _, _ = dg.msd_dataset(900, 0, 8, seed=78)
    hyp = (1.0, 1.0, 0.1)
    with g.GP(X, y, hyp, n_tiles=4) as a:
        ha = a.optimize(6)
    with g.GP(X, y, hyp, n_tiles=4, scheduler="persistent") as p:
        hp = p.optimize(6)
    assert np.array_equal(ha, hp)


def test_persistent_rejected_for_mixed(g):
    X, y, _, _ = dg.msd_dataset(256, 0, 4, seed=79)
    with pytest.raises(g.GPError) as e:
        g.GP(X, y, (1.0, 1.0, 0.1), precision="mixed", scheduler="persistent")
    assert e.value.status == g.GP_ERR_ARG
