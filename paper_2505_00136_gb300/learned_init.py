"""Learned hyperparameter initialiser: corpus, labels, training and evaluation.

Orchestration only: every numeric step runs in the CUDA library (GP
optimisation for the labels, data summaries, the MLP's forward and backward
kernels, its Adam step, inference).  Python generates the seeded synthetic
systems and moves buffers.

Labels are the method's own: for each seeded mass-spring-damper system,
Adam (lr 0.1) on the exact-GP NLML from the default initialisation
(l, nu, sigma^2) = (1, 1, 0.1); the label is log theta after the run.  The
network maps the 64-d summary to those log-hyperparameters and is trained by
full-batch Adam on the mean-squared error.  Its benefit is measured as Adam
steps to reach the default run's best NLML within a relative tolerance.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import time

import numpy as np
import torch

from . import datagen as dg
from . import gprat

DEFAULT_HYPER = (1.0, 1.0, 0.1)


def _ok(st, where):
    if st != gprat.GP_OK:
        raise gprat.GPError(st, -1, where)


def corpus(first_seed: int, count: int, n: int, d: int):
    """`count` seeded random systems (seeds first_seed..), device tensors X (B,n,d), y (B,n)."""
    X, y, prm = dg.msd_corpus(range(first_seed, first_seed + count), n, d)
    return torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), prm


def optimise_runs(X, y, steps, lr=0.1, init=None, n_tiles=4, workers=8, precision="fp64"):
    """Adam runs (one GP handle per system, several CUDA streams in flight).

    Returns (final log theta (B,3) numpy, NLML histories (B, steps) numpy).
    init: None (default hyperparameters) or a (B,3) array of natural-scale starts.
    """
    B = X.shape[0]
    hist = np.empty((B, steps))
    theta = np.empty((B, 3))
    streams = [torch.cuda.Stream() for _ in range(workers)]

    def one(b):
        st = streams[b % workers]
        with torch.cuda.stream(st):
            h0 = DEFAULT_HYPER if init is None else tuple(float(v) for v in init[b])
            with gprat.GP(X[b], y[b], h0, n_tiles=n_tiles, precision=precision,
                          stream=st.cuda_stream) as gp:
                hist[b] = gp.optimize(steps, lr)
                theta[b] = gp.get_state()["log_theta"]

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(one, range(B)))
    return theta, hist


def summaries(X, y, omega):
    """(B, 64) float64 device tensor of data summaries (gp_summary per system)."""
    B, n, d = X.shape
    S = torch.empty((B, 64), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for b in range(B):
        _ok(gprat.gp_summary(X[b].data_ptr(), y[b].data_ptr(), n, d, omega.data_ptr(),
                             S[b].data_ptr(), stream), "gp_summary")
    return S


def new_model(seed=7):
    """He-initialised weights (seeded uniform), zero biases, unit standardisation."""
    m = np.zeros(gprat.GP_MLP_MODEL_FLOATS, dtype=np.float32)
    shapes = [(256, 64), (256, 256), (3, 256)]
    off = 0
    for li, (o, i) in enumerate(shapes):
        lim = np.sqrt(6.0 / i) if li < 2 else np.sqrt(3.0 / i)
        m[off:off + o * i] = dg.uniform(seed, 11 + li, o * i, -lim, lim).astype(np.float32)
        off += o * i + o
    m[gprat.GP_MLP_NPARAM + 64:] = 1.0
    return torch.from_numpy(m).cuda()


def train(S, target, epochs=400, lr=3e-3, seed=7, model=None):
    """Full-batch Adam on the MSE; returns (model, loss history)."""
    B = S.shape[0]
    if model is None:
        model = new_model(seed)
    stream = torch.cuda.current_stream().cuda_stream
    _ok(gprat.gp_mlp_feature_stats(S.data_ptr(), B, model.data_ptr(), stream), "gp_mlp_feature_stats")
    T = torch.as_tensor(target, dtype=torch.float32, device="cuda").contiguous()
    gW = torch.empty(gprat.GP_MLP_NPARAM, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(gW)
    v = torch.zeros_like(gW)
    ws = torch.empty(int(gprat.gp_mlp_workspace_floats(B)), dtype=torch.float32, device="cuda")
    loss = torch.empty(epochs, dtype=torch.float32, device="cuda")
    for t in range(1, epochs + 1):
        _ok(gprat.gp_mlp_loss_grad(model.data_ptr(), S.data_ptr(), T.data_ptr(), B, gW.data_ptr(),
                                   loss[t - 1:].data_ptr(), ws.data_ptr(), stream), "gp_mlp_loss_grad")
        _ok(gprat.gp_mlp_adam(model.data_ptr(), gW.data_ptr(), m.data_ptr(), v.data_ptr(), t, lr,
                              0.9, 0.999, 1e-8, stream), "gp_mlp_adam")
    return model, loss.cpu().numpy()


def predict_init(model, X, y, omega):
    """Natural-scale initial hyperparameters (B,3) from gp_learned_init."""
    B, n, d = X.shape
    scratch = torch.empty(gprat.GP_LEARNED_INIT_SCRATCH, dtype=torch.float64, device="cuda")
    out = np.empty((B, 3))
    hp = gprat.gp_hyper()
    stream = torch.cuda.current_stream().cuda_stream
    for b in range(B):
        _ok(gprat.gp_learned_init(X[b].data_ptr(), y[b].data_ptr(), n, d, model.data_ptr(),
                                  omega.data_ptr(), scratch.data_ptr(), ctypes.byref(hp), stream),
            "gp_learned_init")
        out[b] = (hp.lengthscale, hp.vertical, hp.noise_var)
    return out


def steps_to_reach(hist, target, rtol):
    """First step t (1-based count) whose NLML is within rtol of target or below it,
    NLML_t <= target + rtol |target|; len+1 if never."""
    ok = hist <= target + rtol * np.abs(target)
    idx = np.argmax(ok)
    return int(idx + 1) if ok[idx] else len(hist) + 1


def run(n_train_sys=256, n_eval_sys=32, n=256, n_eval=256, d=32, label_steps=600, eval_steps=2000,
        epochs=600, lr=1e-3, rtol=1e-6, first_seed=20000, precision="fp64", workers=8, n_tiles=4):
    """Corpus -> labels -> training -> evaluation; returns a dict of results.

    Convergence is measured against the default run's own optimum: NLML* = the
    minimum over eval_steps Adam steps (lr 0.1) from the default start.  Steps
    to converge = the first step whose NLML is within rtol of NLML* (or below
    it), for the default and the learned start alike; a learned run that never
    gets there counts eval_steps + 1 (reported as capped).  Whether the default
    run has itself settled is reported as the relative NLML change over its
    last 100 steps."""
    t0 = time.perf_counter()
    omega = torch.from_numpy(dg.rff_frequencies()).cuda()
    Xtr, ytr, _ = corpus(first_seed, n_train_sys, n, d)
    labels, _ = optimise_runs(Xtr, ytr, label_steps, precision=precision, workers=workers, n_tiles=n_tiles)
    t_label = time.perf_counter() - t0
    S = summaries(Xtr, ytr, omega)
    t1 = time.perf_counter()
    model, loss = train(S, labels, epochs=epochs, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    Xev, yev, _ = corpus(first_seed + n_train_sys, n_eval_sys, n_eval, d)
    _, h_def = optimise_runs(Xev, yev, eval_steps, workers=workers, n_tiles=n_tiles)
    init = predict_init(model, Xev, yev, omega)
    _, h_lrn = optimise_runs(Xev, yev, eval_steps, init=init, workers=workers, n_tiles=n_tiles)
    best = h_def.min(axis=1)      # NLML*: the default initialisation's optimum over its run
    s_def = np.array([steps_to_reach(h_def[b], best[b], rtol) for b in range(n_eval_sys)])
    s_lrn = np.array([steps_to_reach(h_lrn[b], best[b], rtol) for b in range(n_eval_sys)])
    tail = min(100, eval_steps - 1)
    settle = np.abs(h_def[:, -1] - h_def[:, -1 - tail]) / np.abs(h_def[:, -1])
    return {"median_steps_default": float(np.median(s_def)), "median_steps_learned": float(np.median(s_lrn)),
            "steps_default": s_def.tolist(), "steps_learned": s_lrn.tolist(),
            "cap": eval_steps, "learned_capped": int(np.sum(s_lrn > eval_steps)),
            "default_last100_rel_change_median": float(np.median(settle)),
            "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
            "label_s": t_label, "train_s": t_train, "total_s": time.perf_counter() - t0,
            "corpus": {"train_systems": n_train_sys, "eval_systems": n_eval_sys, "n_train": n,
                       "n_eval": n_eval, "regressors": d, "label_steps": label_steps,
                       "eval_steps": eval_steps, "epochs": epochs, "rtol": rtol}}
