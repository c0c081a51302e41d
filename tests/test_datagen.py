"""The seeded input generators, pinned on CPU to their published definitions.

Both sides of every parity test draw their inputs from ``datagen``, so a
mistake there would be invisible to parity: these pins hold it to SplitMix64's
reference outputs, to the Box-Muller identity, and the mass-spring-damper
integrator to the closed form of one classical RK4 step on a linear system.
"""
import numpy as np
import pytest

from paper_2505_00136_gb300 import datagen as dg

_M64 = (1 << 64) - 1


def _splitmix64_scalar(seed, count):
    """SplitMix64 as a scalar generator on Python integers: state += golden
    gamma, then the three xor-shift-multiply rounds of the finaliser."""
    out, x = [], seed & _M64
    for _ in range(count):
        x = (x + 0x9E3779B97F4A7C15) & _M64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_reference_outputs_for_seed_zero():
    # The first outputs of the reference splitmix64.c seeded with 0.
    got = [int(v) for v in dg.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("seed", [1, 0x123456789ABCDEF0, _M64])
def test_splitmix64_matches_scalar_generator_and_slices(seed):
    ref = _splitmix64_scalar(seed, 40)
    assert [int(v) for v in dg.splitmix64(seed, 40)] == ref
    # counter-based: any slice regenerates on its own
    assert [int(v) for v in dg.splitmix64(seed, 7, offset=29)] == ref[29:36]


def test_uniform_takes_the_top_53_bits():
    bits = dg.splitmix64(dg.stream_key(5, 2), 1000)
    u = dg.uniform(5, 2, 1000)
    assert np.array_equal(u * 2.0 ** 53, (bits >> np.uint64(11)).astype(np.float64))
    v = dg.uniform(5, 2, 1000, -3.0, 1.0)
    assert np.array_equal(v, -3.0 + 4.0 * u)
    assert v.min() >= -3.0 and v.max() < 1.0


def test_uniform_moments():
    u = dg.uniform(11, 0, 200_000)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 1e-3


def test_normal_is_box_muller_of_the_uniform_stream():
    n = 1001
    z = dg.normal(9, 1, n)
    u = dg.uniform(9, 1, n + 1)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    # each pair (z0, z1) has squared radius -2 log u1 and angle 2 pi u2
    r2 = z[0:n - 1:2] ** 2 + z[1::2] ** 2
    assert np.allclose(r2, -2.0 * np.log(u1[: r2.size]), rtol=1e-12, atol=1e-300)
    ang = np.arctan2(z[1::2], z[0:n - 1:2]) % (2 * np.pi)
    assert np.allclose(ang, (2 * np.pi * u2[: ang.size]) % (2 * np.pi), atol=1e-9)


def test_normal_moments():
    z = dg.normal(3, 4, 400_000)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_streams_and_seeds_are_distinct():
    a = dg.uniform(1, 0, 64)
    assert not np.array_equal(a, dg.uniform(1, 1, 64))
    assert not np.array_equal(a, dg.uniform(2, 0, 64))
    assert np.array_equal(a, dg.uniform(1, 0, 64))


def _rk4_step_matrices(m, c, k, dt):
    """One classical RK4 step on s' = A s + g u (s = (x, x'), u constant over
    the step) is s+ = P(hA) s + h Q(hA) g u with P(z) = 1 + z + z^2/2 + z^3/6
    + z^4/24 and Q(z) = 1 + z/2 + z^2/6 + z^3/24 (Taylor polynomials of exp)."""
    A = np.array([[0.0, 1.0], [-k / m, -c / m]])
    g = np.array([0.0, 1.0 / m])
    Z = dt * A
    I2 = np.eye(2)
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    P = I2 + Z + Z2 / 2 + Z3 / 6 + Z3 @ Z / 24
    Q = I2 + Z / 2 + Z2 / 6 + Z3 / 24
    return P, dt * Q @ g


@pytest.mark.parametrize("m,c,k,dt", [(1.0, 0.5, 2.0, 0.1), (0.7, 0.9, 4.1, 0.05), (1.8, 0.2, 0.6, 0.1)])
def test_msd_integrator_is_the_rk4_step_polynomial(m, c, k, dt):
    u = dg.uniform(21, 0, 300, -1.0, 1.0)
    x = dg.msd_simulate(u, m, c, k, dt)
    P, q = _rk4_step_matrices(m, c, k, dt)
    s = np.zeros(2)
    ref = np.empty(u.size)
    for j in range(u.size):
        ref[j] = s[0]
        s = P @ s + q * u[j]
    assert np.allclose(x, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_msd_step_response_approaches_the_closed_form():
    # Constant input U from rest, underdamped: x(t) = U/k (1 - e^{-zw t}(cos wd t + zw/wd sin wd t)).
    m, c, k, U, dt = 1.0, 0.5, 2.0, 0.7, 0.1
    T = 400
    x = dg.msd_simulate(np.full(T, U), m, c, k, dt)
    w0 = np.sqrt(k / m)
    zw = c / (2 * m)
    wd = np.sqrt(w0 ** 2 - zw ** 2)
    t = dt * np.arange(T)
    exact = U / k * (1 - np.exp(-zw * t) * (np.cos(wd * t) + zw / wd * np.sin(wd * t)))
    assert np.abs(x - exact).max() < 1e-5 * U / k       # RK4 global error O(dt^4)
    assert x[0] == 0.0


def test_msd_is_linear_and_time_invariant():
    u1 = dg.uniform(4, 0, 200, -1.0, 1.0)
    u2 = dg.uniform(4, 1, 200, -1.0, 1.0)
    x1, x2 = dg.msd_simulate(u1, 1.0, 0.5, 2.0), dg.msd_simulate(u2, 1.0, 0.5, 2.0)
    x12 = dg.msd_simulate(2.5 * u1 + u2, 1.0, 0.5, 2.0)
    assert np.allclose(x12, 2.5 * x1 + x2, rtol=0, atol=1e-13)
    shifted = dg.msd_simulate(np.concatenate([[0.0], u1[:-1]]), 1.0, 0.5, 2.0)
    assert np.allclose(shifted[1:], x1[:-1], rtol=0, atol=1e-15)


def test_batched_simulation_matches_single_systems():
    U = np.stack([dg.uniform(s, 0, 120, -1.0, 1.0) for s in (1, 2, 3)])
    prm = np.array([[1.0, 0.5, 2.0], [0.6, 0.3, 4.0], [1.9, 0.9, 0.7]])
    X = dg.msd_simulate(U, prm[:, 0], prm[:, 1], prm[:, 2])
    for b in range(3):
        assert np.array_equal(X[b], dg.msd_simulate(U[b], *prm[b]))


def test_lagged_regressors_layout():
    u = np.arange(1.0, 7.0)
    Z = dg.lagged_regressors(u, 3)
    assert Z.shape == (6, 3)
    assert np.array_equal(Z[0], [0, 0, 0])
    assert np.array_equal(Z[2], [2, 1, 0])
    assert np.array_equal(Z[5], [5, 4, 3])


def test_msd_dataset_split_and_determinism():
    n, m, d = 100, 30, 8
    X, y, Xs, ys = dg.msd_dataset(n, m, d, seed=7)
    assert X.shape == (n, d) and Xs.shape == (m, d) and y.shape == (n,) and ys.shape == (m,)
    assert X.flags.c_contiguous and Xs.flags.c_contiguous
    u = dg.uniform(7, 0, n + m, -1.0, 1.0)
    # the test rows continue the training rows: row j holds u_{j-1} .. u_{j-d}
    assert np.array_equal(X[n - 1], u[n - 2:n - 2 - d:-1])
    assert np.array_equal(Xs[0], u[n - 1:n - 1 - d:-1])
    assert np.array_equal(Xs[0, 1:], X[n - 1, :-1])
    x = dg.msd_simulate(u, 1.0, 0.5, 2.0)
    noise = np.concatenate([y, ys]) - x
    assert np.allclose(noise, 0.1 * dg.normal(7, 1, n + m), rtol=0, atol=1e-15)
    X2, y2, _, _ = dg.msd_dataset(n, m, d, seed=7)
    assert np.array_equal(X, X2) and np.array_equal(y, y2)
