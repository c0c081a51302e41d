"""Learned initialiser: summary and MLP kernels against the FP64 oracle, the
weight-Adam kernel against torch.optim.Adam, and the end-to-end gain over the
default initialisation on held-out systems.
"""
import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg
from _util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_00136_gb300 import build
    build.build()
    from paper_2505_00136_gb300 import gprat, learned_init
    return torch, gprat, learned_init


@pytest.mark.parametrize("n,d", [(300, 32), (257, 12), (1024, 48), (64, 1)])
def test_summary_kernel_matches_oracle(env, orc, n, d):
    torch, gprat, _ = env
    X, y, _, _ = dg.msd_dataset(n, 0, d, seed=60 + d)
    om = dg.rff_frequencies()
    s_o = orc.summary(X, y, om)
    Xd, yd, omd = (torch.from_numpy(a).cuda() for a in (X, y, om))
    s = torch.empty(64, dtype=torch.float64, device="cuda")
    assert gprat.gp_summary(Xd.data_ptr(), yd.data_ptr(), n, d, omd.data_ptr(), s.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert rel(s.cpu().numpy(), s_o) < 1e-12


def _random_model(torch, gprat, seed):
    W = np.concatenate([dg.uniform(seed, 1, gprat.GP_MLP_NPARAM, -0.15, 0.15),
                        np.zeros(64), np.ones(64)]).astype(np.float32)
    return W, torch.from_numpy(W).cuda()


def test_mlp_forward_and_gradient_match_oracle(env, orc):
    torch, gprat, _ = env
    B = 37                                   # several CTAs and a ragged tail
    W, Wd = _random_model(torch, gprat, 3)
    S = dg.uniform(4, 2, B * 64, -1.0, 1.0).reshape(B, 64)
    T = dg.uniform(5, 3, B * 3, -2.0, 2.0).reshape(B, 3)
    Sd = torch.from_numpy(S).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    out = torch.empty(B * 3, dtype=torch.float32, device="cuda")
    assert gprat.gp_mlp_forward(Wd.data_ptr(), Sd.data_ptr(), B, out.data_ptr(), None) == 0
    Wn = W[:gprat.GP_MLP_NPARAM].astype(np.float64)
    o_ref = orc.mlp_forward(Wn, S)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy().reshape(B, 3), o_ref) < 1e-5
    gW = torch.empty(gprat.GP_MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ws = torch.empty(int(gprat.gp_mlp_workspace_floats(B)), dtype=torch.float32, device="cuda")
    assert gprat.gp_mlp_loss_grad(Wd.data_ptr(), Sd.data_ptr(), Td.data_ptr(), B, gW.data_ptr(),
                                  loss.data_ptr(), ws.data_ptr(), None) == 0
    l_ref, g_ref = orc.mlp_loss_grad(Wn, S, T.astype(np.float32).astype(np.float64))
    torch.cuda.synchronize()
    assert abs(loss.item() - l_ref) < 1e-5 * abs(l_ref)
    assert rel(gW.cpu().numpy(), g_ref) < 1e-5


def test_feature_standardisation_is_applied(env, orc):
    torch, gprat, _ = env
    B = 20
    W, Wd = _random_model(torch, gprat, 9)
    S = dg.uniform(8, 2, B * 64, -3.0, 5.0).reshape(B, 64)
    Sd = torch.from_numpy(S).cuda()
    assert gprat.gp_mlp_feature_stats(Sd.data_ptr(), B, Wd.data_ptr(), None) == 0
    out = torch.empty(B * 3, dtype=torch.float32, device="cuda")
    assert gprat.gp_mlp_forward(Wd.data_ptr(), Sd.data_ptr(), B, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    Z = (S - S.mean(0)) / S.std(0)           # numpy statistics, the definition of standardising
    o_ref = orc.mlp_forward(W[:gprat.GP_MLP_NPARAM].astype(np.float64), Z)
    assert rel(out.cpu().numpy().reshape(B, 3), o_ref) < 1e-4


def test_weight_adam_matches_torch_adam(env):
    torch, gprat, _ = env
    W0, Wd = _random_model(torch, gprat, 11)
    p = torch.nn.Parameter(torch.from_numpy(W0[:gprat.GP_MLP_NPARAM].copy()).cuda())
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m = torch.zeros(gprat.GP_MLP_NPARAM, device="cuda")
    v = torch.zeros_like(m)
    for t in range(1, 6):
        g = torch.from_numpy(dg.uniform(12, t, gprat.GP_MLP_NPARAM, -1, 1).astype(np.float32)).cuda()
        p.grad = g.clone()
        opt.step()
        assert gprat.gp_mlp_adam(Wd.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), t, 3e-3, 0.9, 0.999,
                                 1e-8, None) == 0
    torch.cuda.synchronize()
    assert rel(Wd[:gprat.GP_MLP_NPARAM].cpu().numpy(), p.detach().cpu().numpy()) < 1e-6


def test_learned_init_takes_host_or_device_buffers(env):
    """gp_learned_init detects host and device pointers per argument: the
    same data, network and frequencies from host memory (scratch NULL) and
    from device memory give the same hyperparameters."""
    torch, gprat, _ = env
    import ctypes
    X, y, _, _ = dg.msd_dataset(512, 0, 16, seed=77)
    om = dg.rff_frequencies()
    W, Wd = _random_model(torch, gprat, 5)
    Xd, yd, omd = (torch.from_numpy(a).cuda() for a in (X, y, om))
    scratch = torch.empty(gprat.GP_LEARNED_INIT_SCRATCH, dtype=torch.float64, device="cuda")
    hd, hh = gprat.gp_hyper(), gprat.gp_hyper()
    assert gprat.gp_learned_init(Xd.data_ptr(), yd.data_ptr(), 512, 16, Wd.data_ptr(), omd.data_ptr(),
                                 scratch.data_ptr(), ctypes.byref(hd), None) == 0
    Xh, yh, omh = (np.ascontiguousarray(a) for a in (X, y, om))
    assert gprat.gp_learned_init(Xh.ctypes.data, yh.ctypes.data, 512, 16, W.ctypes.data, omh.ctypes.data, None,
                                 ctypes.byref(hh), None) == 0
    a = [hd.lengthscale, hd.vertical, hd.noise_var]
    b = [hh.lengthscale, hh.vertical, hh.noise_var]
    assert all(np.isfinite(a)) and a == b, (a, b)


def test_learned_initialiser_cuts_adam_steps(env):
    """Small corpus (192 systems, n=256, 32 lagged inputs, labels = log theta
    after 600 Adam steps from the default): the trained network's
    initialisation reaches the default run's optimum over 2000 steps (within
    1e-6 relative) in fewer Adam steps, in the median over 24 held-out
    systems, and the default runs have settled by their end."""
    torch, gprat, li = env
    res = li.run(n_train_sys=192, n_eval_sys=24, n=256, n_eval=256, d=32, label_steps=600, eval_steps=2000,
                 epochs=600)
    print("learned init", {k: v for k, v in res.items() if not k.startswith("steps_")})
    assert res["loss_last"] < 0.5 * res["loss_first"]
    assert res["median_steps_default"] < res["cap"]
    assert res["median_steps_learned"] < res["median_steps_default"]
