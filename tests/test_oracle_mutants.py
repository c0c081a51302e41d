"""Each pin must bite: plant a plausible mistake in a copy of the oracle, on the
CPU, and check that the pin suite fails on it.

Mutants cover a dropped term, a wrong sign, a transposed operand or index, a
wrong factor and a wrong parameterisation in every oracle routine the GPU path
is compared with.
"""
import os
import subprocess
import sys

import pytest

import oracle as oracle_mod

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = {
    "noise_term_dropped": ("for (int64_t i = 0; i < n; ++i) K[i * n + i] += hyp[2];", ""),
    "kernel_factor_2": ("/ (2.0 * l * l));\n}", "/ (l * l));\n}"),
    "cholesky_transposed": ("s -= L[i * n + k] * L[j * n + k];", "s -= L[i * n + k] * L[k * n + j];"),
    "forward_sign": ("s -= L[i * n + k] * x[k];", "s += L[i * n + k] * x[k];"),
    "backward_transposed": ("s -= L[k * n + i] * x[k];", "s -= L[i * n + k] * x[k];"),
    "mean_uses_beta": ("s += Kc[i * n + j] * alpha[j];", "s += Kc[i * n + j] * beta[j];"),
    "variance_sign": ("var[i] = prior - s;", "var[i] = prior + s;"),
    "covariance_sign": ("cov[i * m + k] -= s;", "cov[i * m + k] += s;"),
    "nlml_half_dropped": ("return 0.5 * fit + logdet_half", "return fit + logdet_half"),
    "grad_l_factor": ("g_l += w * kf * r2 / (l * l);", "g_l += w * kf * r2 / l;"),
    "grad_noise_delta_dropped": ("if (i == j) g_s2 += w * s2;", "g_s2 += w * s2;"),
    "adam_bias_correction_dropped": ("double mhat = mom[p] / (1.0 - pow(beta1, (double)t));",
                                     "double mhat = mom[p];"),
    "mlp_relu_mask_dropped": ("d2[k] = h2[k] > 0.0 ? a : 0.0;", "d2[k] = a;"),
    "summary_lag_off_by_one": ("c += (y[i] - ybar) * (y[i + lag] - ybar);",
                               "c += (y[i] - ybar) * (y[i + lag - 1] - ybar);"),
    "matern32_linear_term_dropped": ("return nu * (1.0 + s) * exp(-s);", "return nu * exp(-s);"),
    "matern52_dlogl_factor": ("return nu * s * s * (1.0 + s) * exp(-s) / 3.0;",
                              "return nu * s * s * (1.0 + s) * exp(-s);"),
    "matern_squared_distance": ("out[i * nb + j] = matern(kind, sqrt(sqdist(A + i * d, B + j * d, d)), l, nu);",
                                "out[i * nb + j] = matern(kind, sqdist(A + i * d, B + j * d, d), l, nu);"),
    "chol_inverse_transposed": ("s += Linv[k * n + i] * Linv[k * n + j];", "s += Linv[i * n + k] * Linv[j * n + k];"),
    "tri_inverse_row_col": ("for (int64_t i = 0; i < n; ++i) Linv[i * n + c] = col[i];",
                            "for (int64_t i = 0; i < n; ++i) Linv[c * n + i] = col[i];"),
    "logdet_doubled": ("logdet_half += log(L[i * n + i]);", "logdet_half += 2.0 * log(L[i * n + i]);"),
    "nlml_2pi_dropped": (" + 0.5 * (double)n * log(2.0 * M_PI);", ";"),
    "grad_nu_kernel_dropped": ("g_nu += w * kf;", "g_nu += w;"),
    "grad_weight_sign": ("double w = Kinv[i * n + j] - alpha[i] * alpha[j];",
                         "double w = Kinv[i * n + j] + alpha[i] * alpha[j];"),
    "se_nu_dropped_in_gradient": ("kf = nu * exp(-r2 / (2.0 * l * l));", "kf = exp(-r2 / (2.0 * l * l));"),
    "variance_noise_prior_dropped": ("double prior = hyp[1] + (noisy ? hyp[2] : 0.0);", "double prior = hyp[1];"),
    "covariance_noise_dropped": ("if (noisy) cov[i * m + i] += hyp[2];", ""),
    "summary_sample_sd": ("sd[k] = sqrt(v / (double)n);", "sd[k] = sqrt(v / (double)(n - 1));"),
    "summary_sorted_ascending": ("return (x < y) - (x > y);", "return (x > y) - (x < y);"),
    "summary_fourier_swapped": ("s[48 + 2 * q] = cs / (double)n;\n        s[49 + 2 * q] = sn / (double)n;",
                                "s[48 + 2 * q] = sn / (double)n;\n        s[49 + 2 * q] = cs / (double)n;"),
    "summary_acf_uncentred": ("c += (y[i] - ybar) * (y[i + lag] - ybar);", "c += y[i] * y[i + lag];"),
    "mlp_loss_gradient_factor": ("dO[j] = 2.0 * e * scale;", "dO[j] = e * scale;"),
    "mlp_output_bias_dropped": ("double a = W[OFF_B3 + j];", "double a = 0.0;"),
    "adam_eps_inside_sqrt": ("theta[p] -= lr * mhat / (sqrt(vhat) + eps);",
                             "theta[p] -= lr * mhat / sqrt(vhat + eps);"),
    "adam_second_moment_not_squared": ("vel[p] = beta2 * vel[p] + (1.0 - beta2) * g[p] * g[p];",
                                       "vel[p] = beta2 * vel[p] + (1.0 - beta2) * fabs(g[p]);"),
    # Adam on the natural scale instead of log theta: every site of the log/exp map replaced
    "optimize_natural_scale": [
        ("double theta[3] = {log(hyp[0]), log(hyp[1]), log(hyp[2])};", "double theta[3] = {hyp[0], hyp[1], hyp[2]};"),
        ("double h[3] = {exp(theta[0]), exp(theta[1]), exp(theta[2])};", "double h[3] = {theta[0], theta[1], theta[2]};"),
        ("hyp[0] = exp(theta[0]);\n    hyp[1] = exp(theta[1]);\n    hyp[2] = exp(theta[2]);",
         "hyp[0] = theta[0];\n    hyp[1] = theta[1];\n    hyp[2] = theta[2];"),
    ],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    sites = MUTANTS[name]
    if isinstance(sites, tuple):
        sites = [sites]
    src = open(SRC).read()
    for orig, repl in sites:
        assert src.count(orig) == 1, f"mutation site for {name} not unique/present"
        src = src.replace(orig, repl)
    mut_c = tmp_path / "oracle_mut.c"
    mut_c.write_text(src)
    (tmp_path / "oracle.h").write_text(open(os.path.join(os.path.dirname(SRC), "oracle.h")).read())
    lib = oracle_mod.build(str(mut_c), str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, GPRAT_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
