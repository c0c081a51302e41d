"""Thin ctypes binding of the C ABI in ``include/gprat_gb.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libgprat_gb.so``.  Importing this module fails loudly (``ImportError``)
when that library has not been built; there is no CPU fallback.

Buffers may be numpy arrays (host memory) or torch tensors (host or CUDA);
the library detects which from the pointer.  Module-level functions carry the
C names (``gp_create``, ``gp_factor``, ...); :class:`GP` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgprat_gb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library {LIB_PATH} is not built; run paper_2505_00136_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)

GP_OK, GP_ERR_ARG, GP_ERR_NOT_PD, GP_ERR_CUDA, GP_ERR_OOM, GP_ERR_TIMEOUT, GP_ERR_STATE = range(7)
GP_FP64, GP_MIXED, GP_FP64_OZAKI = 0, 1, 2
GP_SCHED_STREAM, GP_SCHED_PERSISTENT = 0, 1
KERNELS = {"se": 0, "matern12": 1, "matern32": 2, "matern52": 3}   # gp_kernel
GP_MLP_NPARAM = 83203
GP_MLP_MODEL_FLOATS = GP_MLP_NPARAM + 128
GP_LEARNED_INIT_SCRATCH = 72
PHASES = ["assemble", "potrf", "trsm", "update", "solve", "cross", "vsolve", "reduce", "cov",
          "trtri", "lauum", "adjoint", "adam", "refine", "bsolve", "ozaki", "rsolve", "slices", "other"]


class gp_hyper(ctypes.Structure):
    _fields_ = [("lengthscale", ctypes.c_double), ("vertical", ctypes.c_double),
                ("noise_var", ctypes.c_double), ("trainable", ctypes.c_int * 3)]


class gp_options(ctypes.Structure):
    _fields_ = [("n_tiles", ctypes.c_int), ("prec", ctypes.c_int), ("noisy_test_var", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("refine_max_iter", ctypes.c_int),
                ("adam_beta1", ctypes.c_double), ("adam_beta2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("scheduler", ctypes.c_int), ("var_correction", ctypes.c_int),
                ("dag_timeout_ms", ctypes.c_int), ("kernel", ctypes.c_int), ("jitter_retries", ctypes.c_int)]


class gp_state(ctypes.Structure):
    _fields_ = [("log_theta", ctypes.c_double * 3), ("adam_m", ctypes.c_double * 3),
                ("adam_v", ctypes.c_double * 3), ("adam_t", ctypes.c_int64)]


class gp_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("tile", ctypes.c_int64),
                ("n_tiles", ctypes.c_int64), ("n_padded", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("refine_iters", ctypes.c_int),
                ("refine_residual", ctypes.c_double), ("jitter_added", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_H = ctypes.c_void_p
_SIGS = {
    "gp_default_options": (None, [ctypes.POINTER(gp_options)]),
    "gp_create": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.POINTER(gp_hyper),
                                 ctypes.POINTER(gp_options), ctypes.POINTER(_H)]),
    "gp_factor": (ctypes.c_int, [_H]),
    "gp_predict": (ctypes.c_int, [_H, _vp, _i64, _vp, _vp, _vp]),
    "gp_predict_mean": (ctypes.c_int, [_H, _vp, _i64, _vp]),
    "gp_predict_var": (ctypes.c_int, [_H, _vp, _i64, _vp, _vp]),
    "gp_predict_full_cov": (ctypes.c_int, [_H, _vp, _i64, _vp, _vp]),
    "gp_nlml": (ctypes.c_int, [_H, _vp]),
    "gp_nlml_grad": (ctypes.c_int, [_H, _vp, _vp]),
    "gp_optimize": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, _vp]),
    "gp_get_hyper": (ctypes.c_int, [_H, ctypes.POINTER(gp_hyper)]),
    "gp_set_hyper": (ctypes.c_int, [_H, ctypes.POINTER(gp_hyper)]),
    "gp_get_state": (ctypes.c_int, [_H, ctypes.POINTER(gp_state)]),
    "gp_set_state": (ctypes.c_int, [_H, ctypes.POINTER(gp_state)]),
    "gp_get_factor": (ctypes.c_int, [_H, _vp]),
    "gp_get_alpha": (ctypes.c_int, [_H, _vp]),
    "gp_dag_stall_tile": (ctypes.c_int, [_H, _i64, _i64]),
    "gp_solve_stall": (ctypes.c_int, [_H, ctypes.c_int, _i64]),
    "gp_info": (ctypes.c_int, [_H, ctypes.POINTER(gp_info_t)]),
    "gp_profile": (ctypes.c_int, [_H, ctypes.c_int]),
    "gp_profile_read": (ctypes.c_int, [_H, _vp, _vp, ctypes.c_int]),
    "gp_launch_count": (_i64, [_H]),
    "gp_auto_tiles": (_i64, [_i64]),
    "gp_predict_mean_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _i64, ctypes.c_double,
                                               ctypes.c_double, _vp, _vp]),
    "gp_summary": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "gp_mlp_feature_stats": (ctypes.c_int, [_vp, _i64, _vp, _vp]),
    "gp_mlp_workspace_floats": (_i64, [_i64]),
    "gp_mlp_forward": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "gp_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gp_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, _vp]),
    "gp_learned_init": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, ctypes.POINTER(gp_hyper), _vp]),
    "gp_measure_fp64_peaks": (ctypes.c_int, [_vp, _vp, _vp]),
    "gp_last_error_info": (_i64, [_H]),
    "gp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "gp_destroy": (None, [_H]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

# Entry points added beside the ones above are declared where they are used.
EXPORTED = sorted(_SIGS)


class GPError(RuntimeError):
    """A C-ABI call returned a status other than GP_OK."""

    def __init__(self, status: int, info: int = -1, where: str = ""):
        msg = _lib.gp_status_str(status).decode()
        super().__init__(f"{where}: {msg} (status {status}, info {info})")
        self.status = status
        self.info = info


def _ptr(a):
    """Raw address of a numpy array or torch tensor (must be contiguous float64)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous and a.dtype == np.float64
        return a.ctypes.data
    # torch.Tensor
    assert a.is_contiguous() and str(a.dtype) == "torch.float64"
    return a.data_ptr()


def _is_torch(a):
    return a is not None and not isinstance(a, np.ndarray) and hasattr(a, "data_ptr")


def _check(status, h=None, where=""):
    if status != GP_OK:
        info = _lib.gp_last_error_info(h) if h else -1
        raise GPError(status, info, where)


def auto_tiles(n: int) -> int:
    """Tiles per dimension chosen for n training points (``gp_auto_tiles``);
    ``GP(..., n_tiles=0)`` uses it."""
    return int(_lib.gp_auto_tiles(int(n)))


def measure_fp64_peaks(stream=None):
    """(DMMA, DFMA) FP64 TFLOP/s of the current GPU (``gp_measure_fp64_peaks``)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.gp_measure_fp64_peaks(ctypes.addressof(a), ctypes.addressof(b), stream), None,
           "gp_measure_fp64_peaks")
    return a.value, b.value


def default_options() -> gp_options:
    o = gp_options()
    _lib.gp_default_options(ctypes.byref(o))
    return o


class GP:
    """One GP handle (``gp_t``).  Outputs are numpy arrays unless ``X`` was a CUDA
    tensor, in which case they are CUDA tensors on the same device."""

    def __init__(self, X, y, hyper=(1.0, 1.0, 0.1), trainable=(1, 1, 1), n_tiles=16,
                 precision="fp64", noisy_test_var=False, stream=None, scheduler="stream",
                 refine_tol=None, refine_max_iter=None, var_correction=True, dag_timeout_ms=None, kernel="se",
                 jitter_retries=0):
        if not _is_torch(X):
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
        self._torch_dev = X.device if _is_torch(X) and X.is_cuda else None
        n, d = X.shape
        opt = default_options()
        opt.n_tiles = int(n_tiles)
        opt.prec = {"fp64": GP_FP64, "mixed": GP_MIXED, "fp64_ozaki": GP_FP64_OZAKI}[precision]
        opt.noisy_test_var = int(bool(noisy_test_var))
        opt.scheduler = GP_SCHED_PERSISTENT if scheduler == "persistent" else GP_SCHED_STREAM
        if refine_tol is not None:
            opt.refine_tol = refine_tol
        if refine_max_iter is not None:
            opt.refine_max_iter = refine_max_iter
        opt.var_correction = int(bool(var_correction))
        if dag_timeout_ms is not None:
            opt.dag_timeout_ms = int(dag_timeout_ms)
        opt.kernel = KERNELS[kernel]
        opt.jitter_retries = int(jitter_retries)
        if stream is None and self._torch_dev is not None:
            import torch
            stream = torch.cuda.current_stream(self._torch_dev).cuda_stream
        opt.cuda_stream = stream
        hp = gp_hyper(float(hyper[0]), float(hyper[1]), float(hyper[2]),
                      (ctypes.c_int * 3)(*[int(bool(t)) for t in trainable]))
        h = _H()
        self._keep = (X, y)
        _check(_lib.gp_create(_ptr(X), _ptr(y), n, d, ctypes.byref(hp), ctypes.byref(opt),
                              ctypes.byref(h)), None, "gp_create")
        self.h = h
        self.n, self.d = n, d

    # -- helpers
    def _out(self, *shape):
        if self._torch_dev is not None:
            import torch
            return torch.empty(*shape, dtype=torch.float64, device=self._torch_dev)
        return np.empty(shape, dtype=np.float64)

    def _in(self, Xs):
        if _is_torch(Xs):
            return Xs.contiguous()
        return np.ascontiguousarray(Xs, dtype=np.float64)

    def close(self):
        if getattr(self, "h", None):
            _lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C calls
    def factor(self):
        _check(_lib.gp_factor(self.h), self.h, "gp_factor")

    def predict_mean(self, Xs):
        Xs = self._in(Xs)
        mean = self._out(Xs.shape[0])
        _check(_lib.gp_predict_mean(self.h, _ptr(Xs), Xs.shape[0], _ptr(mean)), self.h, "gp_predict_mean")
        return mean

    def predict_var(self, Xs):
        Xs = self._in(Xs)
        m = Xs.shape[0]
        mean, var = self._out(m), self._out(m)
        _check(_lib.gp_predict_var(self.h, _ptr(Xs), m, _ptr(mean), _ptr(var)), self.h, "gp_predict_var")
        return mean, var

    def predict(self, Xs, mean=True, var=True, cov=False):
        """One solve for any of mean, variance and full covariance (``gp_predict``)."""
        Xs = self._in(Xs)
        m = Xs.shape[0]
        mu = self._out(m) if mean else None
        va = self._out(m) if var else None
        cv = self._out(m, m) if cov else None
        _check(_lib.gp_predict(self.h, _ptr(Xs), m, _ptr(mu), _ptr(va), _ptr(cv)), self.h, "gp_predict")
        return mu, va, cv

    def profile(self, enable=True):
        _check(_lib.gp_profile(self.h, int(bool(enable))), self.h, "gp_profile")

    def profile_read(self):
        """Per-phase (ms, launches) accumulated since the last read."""
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), dtype=np.int64)
        _check(_lib.gp_profile_read(self.h, ms.ctypes.data, cnt.ctypes.data, len(PHASES)), self.h,
               "gp_profile_read")
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def launch_count(self):
        return int(_lib.gp_launch_count(self.h))

    def predict_full_cov(self, Xs):
        Xs = self._in(Xs)
        m = Xs.shape[0]
        mean, cov = self._out(m), self._out(m, m)
        _check(_lib.gp_predict_full_cov(self.h, _ptr(Xs), m, _ptr(mean), _ptr(cov)), self.h,
               "gp_predict_full_cov")
        return mean, cov

    def nlml(self):
        out = ctypes.c_double()
        _check(_lib.gp_nlml(self.h, ctypes.addressof(out)), self.h, "gp_nlml")
        return out.value

    def nlml_grad(self):
        f = ctypes.c_double()
        g = (ctypes.c_double * 3)()
        _check(_lib.gp_nlml_grad(self.h, ctypes.addressof(f), ctypes.addressof(g)), self.h, "gp_nlml_grad")
        return f.value, np.array(g[:])

    def optimize(self, steps, lr=0.1):
        hist = np.empty(steps)
        _check(_lib.gp_optimize(self.h, int(steps), float(lr), hist.ctypes.data if steps else None),
               self.h, "gp_optimize")
        return hist

    def get_hyper(self):
        hp = gp_hyper()
        _check(_lib.gp_get_hyper(self.h, ctypes.byref(hp)), self.h, "gp_get_hyper")
        return (hp.lengthscale, hp.vertical, hp.noise_var), tuple(hp.trainable)

    def set_hyper(self, hyper, trainable=(1, 1, 1)):
        hp = gp_hyper(float(hyper[0]), float(hyper[1]), float(hyper[2]),
                      (ctypes.c_int * 3)(*[int(bool(t)) for t in trainable]))
        _check(_lib.gp_set_hyper(self.h, ctypes.byref(hp)), self.h, "gp_set_hyper")

    def get_state(self):
        st = gp_state()
        _check(_lib.gp_get_state(self.h, ctypes.byref(st)), self.h, "gp_get_state")
        return {"log_theta": np.array(st.log_theta[:]), "adam_m": np.array(st.adam_m[:]),
                "adam_v": np.array(st.adam_v[:]), "adam_t": int(st.adam_t)}

    def set_state(self, state):
        st = gp_state((ctypes.c_double * 3)(*state["log_theta"]), (ctypes.c_double * 3)(*state["adam_m"]),
                      (ctypes.c_double * 3)(*state["adam_v"]), int(state["adam_t"]))
        _check(_lib.gp_set_state(self.h, ctypes.byref(st)), self.h, "gp_set_state")

    def get_factor(self):
        L = self._out(self.n, self.n)
        _check(_lib.gp_get_factor(self.h, _ptr(L)), self.h, "gp_get_factor")
        return L

    def get_alpha(self):
        a = self._out(self.n)
        _check(_lib.gp_get_alpha(self.h, _ptr(a)), self.h, "gp_get_alpha")
        return a

    def dag_stall_tile(self, i, j=0):
        """Testing aid: poison tile (i, j)'s update counter (i < 0 clears)."""
        _check(_lib.gp_dag_stall_tile(self.h, int(i), int(j)), self.h, "gp_dag_stall_tile")

    def solve_stall(self, enable, wait_us=0):
        """Testing aid: the mixed path's persistent solves stall at their first
        grid barrier, whose waits are bounded by wait_us (enable=False clears)."""
        _check(_lib.gp_solve_stall(self.h, 1 if enable else 0, int(wait_us)), self.h, "gp_solve_stall")

    def info(self):
        inf = gp_info_t()
        _check(_lib.gp_info(self.h, ctypes.byref(inf)), self.h, "gp_info")
        return {k: getattr(inf, k) for k, _ in gp_info_t._fields_}
