"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call is made here (no GPU): only argument validation that returns
before any CUDA call.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_00136_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ["gp_create", "gp_factor", "gp_predict_mean", "gp_predict_var",
                     "gp_predict_full_cov", "gp_nlml", "gp_nlml_grad", "gp_optimize", "gp_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_declares_same_names(lib):
    from paper_2505_00136_gb300 import gprat
    for n in declared_functions():
        assert hasattr(gprat, n), n


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    from paper_2505_00136_gb300 import gprat as g
    X = np.zeros((4, 2))
    y = np.zeros(4)
    h = g._H()
    hp = g.gp_hyper(1.0, 1.0, 0.1, (ctypes.c_int * 3)(1, 1, 1))
    opt = g.default_options()
    assert opt.n_tiles == 16 and opt.adam_beta1 == 0.9
    px, py = X.ctypes.data, y.ctypes.data
    calls = [
        (None, py, 4, 2, hp, opt),          # NULL X
        (px, py, 0, 2, hp, opt),            # n < 1
        (px, py, 4, 0, hp, opt),            # d < 1
        (px, py, 4, 2000, hp, opt),         # d > 1024
    ]
    for args in calls:
        st = g.gp_create(args[0], args[1], args[2], args[3], ctypes.byref(args[4]),
                         ctypes.byref(args[5]), ctypes.byref(h))
        assert st == g.GP_ERR_ARG
    bad = g.gp_hyper(-1.0, 1.0, 0.1, (ctypes.c_int * 3)(1, 1, 1))
    assert g.gp_create(px, py, 4, 2, ctypes.byref(bad), ctypes.byref(opt), ctypes.byref(h)) == g.GP_ERR_ARG
    opt.n_tiles = -1                        # 0 selects gp_auto_tiles; negative is invalid
    assert g.gp_create(px, py, 4, 2, ctypes.byref(hp), ctypes.byref(opt), ctypes.byref(h)) == g.GP_ERR_ARG
    assert g.gp_factor(None) == g.GP_ERR_ARG
    assert g.gp_solve_stall(None, 1, 1000) == g.GP_ERR_ARG
    assert g.gp_dag_stall_tile(None, 0, 0) == g.GP_ERR_ARG
    assert g.gp_status_str(g.GP_ERR_NOT_PD) == b"matrix not positive definite"


def test_auto_tiles_gives_tiles_of_256(lib):
    """Automatic tile count: T = ceil(n / 256), the tile edge measured fastest
    on GB300 for both precisions (host logic only)."""
    from paper_2505_00136_gb300 import gprat as g
    for n, t in [(0, 0), (-5, 0), (1, 1), (256, 1), (257, 2), (1024, 4), (8192, 32), (32768, 128),
                 (65536, 256), (100000, 391)]:
        assert g.auto_tiles(n) == t, (n, g.auto_tiles(n))
    for n in range(1, 3000, 37):
        t = g.auto_tiles(n)
        b = -(-n // t)                      # tile edge gp_create derives before rounding up
        assert b <= 256 and (t == 1 or -(-n // (t - 1)) > 256)


def test_kernel_and_precision_options_are_validated(lib):
    """An unknown kernel or precision is refused by gp_create before any CUDA call."""
    from paper_2505_00136_gb300 import gprat
    X = np.zeros((64, 2))
    y = np.zeros(64)
    hp = gprat.gp_hyper(1.0, 1.0, 0.1, (ctypes.c_int * 3)(1, 1, 1))
    for field, bad in (("kernel", 7), ("kernel", -1), ("prec", 3)):
        opt = gprat.default_options()
        assert opt.kernel == gprat.KERNELS["se"]
        setattr(opt, field, bad)
        h = ctypes.c_void_p()
        st = gprat.gp_create(X.ctypes.data, y.ctypes.data, 64, 2, ctypes.byref(hp), ctypes.byref(opt),
                             ctypes.byref(h))
        assert st == gprat.GP_ERR_ARG and not h.value


def test_other_entry_points_refuse_bad_arguments_before_any_cuda_call(lib):
    """NULL buffers, empty or oversize problems and invalid options are refused
    with GP_ERR_ARG by every other entry point, before any device work."""
    from paper_2505_00136_gb300 import gprat as g
    X = np.zeros((8, 2))
    y = np.zeros(8)
    px, py = X.ctypes.data, y.ctypes.data
    hp = g.gp_hyper(1.0, 1.0, 0.1, (ctypes.c_int * 3)(1, 1, 1))
    out = g.gp_hyper()
    h = g._H()
    # scheduler and DAG options
    for field, bad in (("scheduler", 2), ("scheduler", -1), ("dag_timeout_ms", -5)):
        opt = g.default_options()
        setattr(opt, field, bad)
        assert g.gp_create(px, py, 8, 2, ctypes.byref(hp), ctypes.byref(opt), ctypes.byref(h)) == g.GP_ERR_ARG
    opt = g.default_options()
    opt.scheduler = g.GP_SCHED_PERSISTENT        # the persistent DAG kernel is FP64 only
    opt.prec = g.GP_MIXED
    assert g.gp_create(px, py, 8, 2, ctypes.byref(hp), ctypes.byref(opt), ctypes.byref(h)) == g.GP_ERR_ARG
    # hyperparameters: nu must be positive, sigma^2 non-negative
    for bad in ((1.0, 0.0, 0.1), (1.0, 1.0, -0.1), (0.0, 1.0, 0.1)):
        bh = g.gp_hyper(*bad, (ctypes.c_int * 3)(1, 1, 1))
        assert g.gp_create(px, py, 8, 2, ctypes.byref(bh), None, ctypes.byref(h)) == g.GP_ERR_ARG
    assert g.gp_create(px, py, 8, 2, ctypes.byref(hp), None, None) == g.GP_ERR_ARG
    # calls on a NULL handle
    d = ctypes.c_double()
    for st in (g.gp_predict_mean(None, px, 4, px), g.gp_predict_var(None, px, 4, px, px),
               g.gp_predict_full_cov(None, px, 4, px, px), g.gp_predict(None, px, 4, px, None, None),
               g.gp_nlml(None, ctypes.byref(d)), g.gp_optimize(None, 1, 0.1, None),
               g.gp_get_hyper(None, ctypes.byref(out)), g.gp_set_hyper(None, ctypes.byref(hp)),
               g.gp_get_factor(None, px), g.gp_get_alpha(None, px)):
        assert st == g.GP_ERR_ARG
    # learned initialiser and its training calls
    assert g.gp_learned_init(None, py, 8, 2, px, px, None, ctypes.byref(out), None) == g.GP_ERR_ARG
    assert g.gp_learned_init(px, py, 1, 2, px, px, None, ctypes.byref(out), None) == g.GP_ERR_ARG
    assert g.gp_learned_init(px, py, 8, 0, px, px, None, ctypes.byref(out), None) == g.GP_ERR_ARG
    assert g.gp_summary(None, py, 8, 2, px, px, None) == g.GP_ERR_ARG
    assert g.gp_summary(px, py, 1, 2, px, px, None) == g.GP_ERR_ARG
    assert g.gp_mlp_forward(px, px, 0, px, None) == g.GP_ERR_ARG
    assert g.gp_mlp_adam(px, px, px, px, 0, 0.1, 0.9, 0.999, 1e-8, None) == g.GP_ERR_ARG
    assert g.gp_mlp_adam(px, px, px, px, 1, 0.0, 0.9, 0.999, 1e-8, None) == g.GP_ERR_ARG
    assert g.gp_mlp_workspace_floats(0) == 0
    assert g.gp_mlp_workspace_floats(17) == 2 * (g.GP_MLP_NPARAM + 1)   # 16 samples per block
    # allocation-free mean: sizes (at most GP_NOALLOC_MAX_TEST = 32768 test points) and hyperparameters
    for args in ((None, px, 8, 2, px, 4, 1.0, 1.0), (px, px, 0, 2, px, 4, 1.0, 1.0),
                 (px, px, 8, 2, px, 0, 1.0, 1.0), (px, px, 8, 2, px, 32768 + 1, 1.0, 1.0),
                 (px, px, 8, 2, px, 4, float("nan"), 1.0), (px, px, 8, 2, px, 4, 1.0, -1.0)):
        assert g.gp_predict_mean_noalloc(*args, px, None) == g.GP_ERR_ARG


def test_binding_fails_loudly_without_the_library(tmp_path):
    """The binding has no CPU fallback: a copy of it next to no built library
    raises ImportError on import."""
    import importlib.util
    import shutil
    src = os.path.join(ROOT, "paper_2505_00136_gb300", "gprat.py")
    shutil.copy(src, tmp_path / "gprat.py")
    spec = importlib.util.spec_from_file_location("gprat_without_library", str(tmp_path / "gprat.py"))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="not built"):
        spec.loader.exec_module(mod)


def test_options_struct_layout_matches_the_binding(lib):
    """gp_default_options writes exactly the binding's gp_options: every field
    gets its default and no byte past the struct is touched."""
    from paper_2505_00136_gb300 import gprat as g
    size = ctypes.sizeof(g.gp_options)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    g.gp_default_options(ctypes.cast(buf, ctypes.POINTER(g.gp_options)))
    assert bytes(buf[size:]) == b"\xab" * 64
    opt = g.gp_options.from_buffer(buf)
    assert (opt.n_tiles, opt.prec, opt.noisy_test_var, opt.refine_max_iter) == (16, g.GP_FP64, 0, 20)
    assert (opt.refine_tol, opt.adam_beta1, opt.adam_beta2, opt.adam_eps) == (1e-14, 0.9, 0.999, 1e-8)
    assert (opt.scheduler, opt.var_correction, opt.dag_timeout_ms) == (g.GP_SCHED_STREAM, 1, 10000)
    assert (opt.kernel, opt.jitter_retries) == (g.KERNELS["se"], 0)
    assert opt.cuda_stream is None


def test_jitter_retries_option_is_validated(lib):
    from paper_2505_00136_gb300 import gprat as g
    X = np.zeros((8, 2))
    y = np.zeros(8)
    hp = g.gp_hyper(1.0, 1.0, 0.1, (ctypes.c_int * 3)(1, 1, 1))
    for bad in (-1, 9):
        opt = g.default_options()
        opt.jitter_retries = bad
        h = g._H()
        assert g.gp_create(X.ctypes.data, y.ctypes.data, 8, 2, ctypes.byref(hp), ctypes.byref(opt),
                           ctypes.byref(h)) == g.GP_ERR_ARG
