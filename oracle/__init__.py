"""ctypes wrapper of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg, never by the product package.  ``build()``
compiles ``oracle.c`` with gcc into ``liboracle.so`` beside it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(src: str = _SRC, out: str = LIB_PATH, extra=()) -> str:
    """Compile the oracle (plain C, -O2, no fast-math, single thread)."""
    cmd = ["gcc", "-std=gnu11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", out, src, "-lm", *extra]
    subprocess.run(cmd, check=True, cwd=_HERE)
    return out


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    return os.path.getmtime(LIB_PATH) < max(os.path.getmtime(_SRC),
                                            os.path.getmtime(os.path.join(_HERE, "oracle.h")))


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def load(path: str | None = None):
    """Load (building first if needed) and declare the oracle's C signatures."""
    global _lib
    if path is None:
        if _lib is not None:
            return _lib
        if _stale():
            build()
        path = LIB_PATH
    lib = ctypes.CDLL(path)
    sig = {
        "orc_version": (ctypes.c_int, []),
        "orc_se_cross": (None, [_D, _i64, _D, _i64, _i64, ctypes.c_double, ctypes.c_double, _D]),
        "orc_cov_train": (None, [_D, _i64, _i64, _D, _D]),
        "orc_cholesky": (_i64, [_D, _i64, _D]),
        "orc_forward": (None, [_D, _i64, _D]),
        "orc_backward": (None, [_D, _i64, _D]),
        "orc_tri_inverse": (None, [_D, _i64, _D]),
        "orc_chol_inverse": (None, [_D, _i64, _D]),
        "orc_predict": (_i64, [_D, _D, _i64, _i64, _D, _i64, _D, ctypes.c_int, _D, _D, _D]),
        "orc_nlml": (_i64, [_D, _D, _i64, _i64, _D, _D]),
        "orc_nlml_grad": (_i64, [_D, _D, _i64, _i64, _D, _D, _D]),
        "orc_adam": (None, [_D, _D, _D, _D, _i64, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, _I]),
        "orc_optimize": (_i64, [_D, _D, _i64, _i64, _D, _I, _i64, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]),
        "orc_kernel_cross": (None, [ctypes.c_int, _D, _i64, _D, _i64, _i64, ctypes.c_double, ctypes.c_double,
                                    _D]),
        "orc_cov_train_k": (None, [ctypes.c_int, _D, _i64, _i64, _D, _D]),
        "orc_predict_k": (_i64, [ctypes.c_int, _D, _D, _i64, _i64, _D, _i64, _D, ctypes.c_int, _D, _D, _D]),
        "orc_nlml_k": (_i64, [ctypes.c_int, _D, _D, _i64, _i64, _D, _D]),
        "orc_nlml_grad_k": (_i64, [ctypes.c_int, _D, _D, _i64, _i64, _D, _D, _D]),
        "orc_optimize_k": (_i64, [ctypes.c_int, _D, _D, _i64, _i64, _D, _I, _i64, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]),
        "orc_summary": (None, [_D, _D, _i64, _i64, _D, _D]),
        "orc_mlp_forward": (None, [_D, _i64, _D, _D]),
        "orc_mlp_loss_grad": (ctypes.c_double, [_D, _i64, _D, _D, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleNotPD(RuntimeError):
    """The oracle met a non-positive pivot; ``row`` is its 0-based index."""

    def __init__(self, row):
        super().__init__(f"matrix not positive definite at row {row}")
        self.row = int(row)


KERNELS = {"se": 0, "matern12": 1, "matern32": 2, "matern52": 3}


class Oracle:
    """Numpy-facing view of one oracle library (the default, or a test-built variant).

    ``kernel`` selects the covariance function: "se" (Eq. 2, the default) or
    the Matern kernels "matern12", "matern32", "matern52"."""

    MLP_NPARAM = 256 * 64 + 256 + 256 * 256 + 256 + 3 * 256 + 3

    def __init__(self, path: str | None = None):
        self.lib = load(path)

    @staticmethod
    def _hyp(hyp):
        return _f64(np.asarray(hyp, dtype=np.float64).reshape(3))

    def se_cross(self, A, B, l, nu):
        A, B = _f64(A), _f64(B)
        out = np.empty((A.shape[0], B.shape[0]))
        self.lib.orc_se_cross(_p(A), A.shape[0], _p(B), B.shape[0], A.shape[1], l, nu, _p(out))
        return out

    def kernel_cross(self, A, B, l, nu, kernel="se"):
        A, B = _f64(A), _f64(B)
        out = np.empty((A.shape[0], B.shape[0]))
        self.lib.orc_kernel_cross(KERNELS[kernel], _p(A), A.shape[0], _p(B), B.shape[0], A.shape[1], l, nu,
                                  _p(out))
        return out

    def cov_train(self, X, hyp, kernel="se"):
        X = _f64(X)
        n = X.shape[0]
        K = np.empty((n, n))
        self.lib.orc_cov_train_k(KERNELS[kernel], _p(X), n, X.shape[1], _p(self._hyp(hyp)), _p(K))
        return K

    def cholesky(self, K):
        K = _f64(K)
        n = K.shape[0]
        L = np.empty((n, n))
        info = self.lib.orc_cholesky(_p(K), n, _p(L))
        if info >= 0:
            raise OracleNotPD(info)
        return L

    def forward(self, L, b):
        L, x = _f64(L), _f64(b).copy()
        self.lib.orc_forward(_p(L), L.shape[0], _p(x))
        return x

    def backward(self, L, b):
        L, x = _f64(L), _f64(b).copy()
        self.lib.orc_backward(_p(L), L.shape[0], _p(x))
        return x

    def tri_inverse(self, L):
        L = _f64(L)
        out = np.empty_like(L)
        self.lib.orc_tri_inverse(_p(L), L.shape[0], _p(out))
        return out

    def chol_inverse(self, L):
        L = _f64(L)
        out = np.empty_like(L)
        self.lib.orc_chol_inverse(_p(L), L.shape[0], _p(out))
        return out

    def predict(self, X, y, Xs, hyp, noisy=False, mean=True, var=True, cov=False, kernel="se"):
        X, y, Xs = _f64(X), _f64(y), _f64(Xs)
        n, d = X.shape
        m = Xs.shape[0]
        mu = np.empty(m) if mean else None
        va = np.empty(m) if var else None
        cv = np.empty((m, m)) if cov else None
        info = self.lib.orc_predict_k(KERNELS[kernel], _p(X), _p(y), n, d, _p(Xs), m, _p(self._hyp(hyp)),
                                      int(bool(noisy)), _p(mu), _p(va), _p(cv))
        if info >= 0:
            raise OracleNotPD(info)
        return mu, va, cv

    def nlml(self, X, y, hyp, kernel="se"):
        X, y = _f64(X), _f64(y)
        out = np.zeros(1)
        info = self.lib.orc_nlml_k(KERNELS[kernel], _p(X), _p(y), X.shape[0], X.shape[1], _p(self._hyp(hyp)),
                                   _p(out))
        if info >= 0:
            raise OracleNotPD(info)
        return float(out[0])

    def nlml_grad(self, X, y, hyp, kernel="se"):
        X, y = _f64(X), _f64(y)
        f = np.zeros(1)
        g = np.zeros(3)
        info = self.lib.orc_nlml_grad_k(KERNELS[kernel], _p(X), _p(y), X.shape[0], X.shape[1],
                                        _p(self._hyp(hyp)), _p(f), _p(g))
        if info >= 0:
            raise OracleNotPD(info)
        return float(f[0]), g

    def adam(self, theta, mom, vel, g, t, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8,
             trainable=(1, 1, 1)):
        th, mo, ve = _f64(theta).copy(), _f64(mom).copy(), _f64(vel).copy()
        tr = np.ascontiguousarray(trainable, dtype=np.int32)
        self.lib.orc_adam(_p(th), _p(mo), _p(ve), _p(_f64(g)), int(t), lr, beta1, beta2, eps,
                          tr.ctypes.data_as(_I))
        return th, mo, ve

    def optimize(self, X, y, hyp, steps, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8,
                 trainable=(1, 1, 1), kernel="se"):
        X, y = _f64(X), _f64(y)
        h = self._hyp(hyp).copy()
        hist = np.empty(steps)
        tr = np.ascontiguousarray(trainable, dtype=np.int32)
        info = self.lib.orc_optimize_k(KERNELS[kernel], _p(X), _p(y), X.shape[0], X.shape[1], _p(h),
                                       tr.ctypes.data_as(_I), steps, lr, beta1, beta2, eps, _p(hist))
        if info >= 0:
            raise OracleNotPD(info)
        return h, hist

    def summary(self, X, y, omega):
        X, y, om = _f64(X), _f64(y), _f64(omega)
        s = np.empty(64)
        self.lib.orc_summary(_p(X), _p(y), X.shape[0], X.shape[1], _p(om), _p(s))
        return s

    def mlp_forward(self, W, S):
        W, S = _f64(W), _f64(S)
        out = np.empty((S.shape[0], 3))
        self.lib.orc_mlp_forward(_p(W), S.shape[0], _p(S), _p(out))
        return out

    def mlp_loss_grad(self, W, S, T):
        W, S, T = _f64(W), _f64(S), _f64(T)
        g = np.empty(self.MLP_NPARAM)
        loss = self.lib.orc_mlp_loss_grad(_p(W), S.shape[0], _p(S), _p(T), _p(g))
        return float(loss), g
