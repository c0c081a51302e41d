"""The allocation-free predictive mean, for callers that cannot allocate device
memory (fixed memory pools, loops that must not enter the allocator, hosts
that forbid allocation).

gp_predict_mean_noalloc is called through the C ABI on caller-owned device
buffers and compared with the handle-based gp_predict_mean on the same inputs,
at the suite's FP64 tolerance, on two calls in a row (different sizes, so the
second call runs on scratch the first one left behind).  Collected last so a
stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import rel

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat
    return torch, gprat


def reference_mean(gprat, torch, X, y, Xs, hyp):
    """mean and alpha from the handle-based path (gp_get_alpha, gp_predict_mean)."""
    Xd, yd, Xsd = (torch.from_numpy(a).cuda() for a in (X, y, Xs))
    with gprat.GP(Xd, yd, hyp, n_tiles=8) as gp:
        alpha = gp.get_alpha()
        mean = gp.predict_mean(Xsd)
        torch.cuda.synchronize()
    return Xd, Xsd, alpha, mean


def call_noalloc(gprat, torch, Xd, alpha, Xsd, hyp, out):
    n, d = Xd.shape
    m = Xsd.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    return gprat.gp_predict_mean_noalloc(Xd.data_ptr(), alpha.data_ptr(), n, d, Xsd.data_ptr(), m,
                                         float(hyp[0]), float(hyp[1]), out.data_ptr(), stream)


def test_noalloc_mean_matches_handle_mean_on_two_calls(env):
    torch, gprat = env
    cases = [((3000, 777, 8, 31), (1.0, 1.0, 0.1)), ((1500, 200, 5, 32), (0.8, 1.3, 0.05))]
    for (n, m, d, seed), hyp in cases:
        X, y, Xs, _ = dg.msd_dataset(n, m, d, seed)
        Xd, Xsd, alpha, ref = reference_mean(gprat, torch, X, y, Xs, hyp)
        out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        st = call_noalloc(gprat, torch, Xd, alpha, Xsd, hyp, out)
        assert st == gprat.GP_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref.cpu().numpy()) < TOL


def test_noalloc_rejects_oversize_and_host_buffers(env):
    torch, gprat = env
    X, y, Xs, _ = dg.msd_dataset(256, 8, 3, 33)
    hyp = (1.0, 1.0, 0.1)
    Xd, Xsd, alpha, _ = reference_mean(gprat, torch, X, y, Xs, hyp)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    too_many = gprat.gp_predict_mean_noalloc(Xd.data_ptr(), alpha.data_ptr(), 256, 3, Xsd.data_ptr(),
                                             gprat_max_test(gprat) + 1, 1.0, 1.0, out.data_ptr(), None)
    assert too_many == gprat.GP_ERR_ARG
    host_out = np.empty(8)
    assert gprat.gp_predict_mean_noalloc(Xd.data_ptr(), alpha.data_ptr(), 256, 3, Xsd.data_ptr(), 8, 1.0, 1.0,
                                         host_out.ctypes.data, None) == gprat.GP_ERR_ARG
    pinned = torch.empty(8, dtype=torch.float64).pin_memory()
    assert gprat.gp_predict_mean_noalloc(Xd.data_ptr(), alpha.data_ptr(), 256, 3, Xsd.data_ptr(), 8, 1.0, 1.0,
                                         pinned.data_ptr(), None) == gprat.GP_ERR_ARG
    if torch.cuda.device_count() > 1:   # a buffer on another GPU is refused before any launch
        other = torch.empty(8, dtype=torch.float64, device="cuda:1")
        assert gprat.gp_predict_mean_noalloc(Xd.data_ptr(), alpha.data_ptr(), 256, 3, Xsd.data_ptr(), 8, 1.0,
                                             1.0, other.data_ptr(), None) == gprat.GP_ERR_ARG


def gprat_max_test(gprat):
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gprat_gb.h")
    return int(re.search(r"#define GP_NOALLOC_MAX_TEST (\d+)", open(hdr).read()).group(1))
