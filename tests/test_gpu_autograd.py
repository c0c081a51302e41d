"""Training through torch.autograd with the hand-written adjoint kernel.

N = 8192 with 8 and 128 lagged regressors, log-parameterised theta: gradient
against central finite differences (h = 1e-5) of the library's own NLML at
1e-6 relative, and against the FP64 oracle at a size it can factor; 50 Adam
steps (lr 0.1) of torch.optim.Adam over the autograd Function against the
library's device-side Adam.
"""
import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import autograd, gprat
    return torch, gprat, autograd


def test_autograd_gradient_matches_oracle(mods, orc):
    torch, gprat, ag = mods
    X, y, _, _ = dg.msd_dataset(1024, 0, 8, seed=1004)
    hyp = (0.9, 1.1, 0.08)
    f_o, g_o = orc.nlml_grad(X, y, hyp)
    with gprat.GP(X, y, hyp, n_tiles=4) as gp:
        th = torch.tensor(np.log(hyp), dtype=torch.float64, requires_grad=True)
        f = ag.nlml(th, gp)
        f.backward()
        assert abs(f.item() - f_o) < 1e-9 * abs(f_o)
        assert max_rel(th.grad.numpy(), g_o, 1e-8 * np.linalg.norm(g_o)) < 1e-9
        # grad_out scaling flows through
        th2 = torch.tensor(np.log(hyp), dtype=torch.float64, requires_grad=True)
        (3.0 * ag.nlml(th2, gp)).backward()
        assert max_rel(th2.grad.numpy(), 3.0 * g_o, 1e-8 * np.linalg.norm(g_o)) < 1e-9


@pytest.mark.parametrize("d,hyp", [(8, (1.0, 1.0, 0.1)), (128, (np.sqrt(128.0), 1.0, 0.1))])
def test_n8192_gradient_vs_central_differences(mods, d, hyp):
    torch, gprat, ag = mods
    X, y, _, _ = dg.msd_dataset(8192, 0, d, seed=1004)
    with gprat.GP(X, y, hyp, n_tiles=32) as gp:
        th = torch.tensor(np.log(hyp), dtype=torch.float64, requires_grad=True)
        ag.nlml(th, gp).backward()
        g = th.grad.numpy()
        h = 1e-5
        fd = np.empty(3)
        for p in range(3):
            v = []
            for s in (1.0, -1.0):
                t = np.log(hyp).copy()
                t[p] += s * h
                gp.set_hyper(np.exp(t))
                v.append(gp.nlml())
            fd[p] = (v[0] - v[1]) / (2 * h)
        assert max_rel(g, fd, 1e-8 * np.linalg.norm(fd)) < 1e-6, (g, fd)


def test_torch_adam_over_autograd_matches_device_adam(mods):
    torch, gprat, ag = mods
    X, y, _, _ = dg.msd_dataset(8192, 0, 8, seed=1004)
    hyp = (1.0, 1.0, 0.1)
    steps = 50
    with gprat.GP(X, y, hyp, n_tiles=32) as gp:
        th = torch.tensor(np.log(hyp), dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([th], lr=0.1, betas=(0.9, 0.999), eps=1e-8)
        hist_torch = []
        for _ in range(steps):
            opt.zero_grad()
            f = ag.nlml(th, gp)
            f.backward()
            opt.step()
            hist_torch.append(f.item())
        th_torch = th.detach().numpy().copy()
    with gprat.GP(X, y, hyp, n_tiles=32) as gp:
        hist_dev = gp.optimize(steps, lr=0.1)
        th_dev = gp.get_state()["log_theta"]
    assert max_rel(hist_torch, hist_dev) < 1e-9
    assert max_rel(th_torch, th_dev) < 1e-8
    assert hist_dev[-1] < hist_dev[0]
