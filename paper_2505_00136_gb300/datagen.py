"""Seeded synthetic inputs shared by the GPU path's tests and by the oracle's tests.

This module produces *inputs* only: it holds none of the Gaussian-process
arithmetic (no kernel, no factorisation, no likelihood).  Both sides of every
parity test draw their data from here, so the oracle and the CUDA path see the
same bits.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser constants
of Vigna's public-domain splitmix64.c).  Value ``i`` of stream ``key`` is the
finaliser applied to ``key + (i + 1) * golden``, i.e. exactly the sequence of a
SplitMix64 generator seeded with ``key``; it is counter-based, so any slice can
be regenerated independently.  Uniform doubles take the top 53 bits; normals
use the Box-Muller transform (Box & Muller 1958).

The workload is the paper's system-identification benchmark (Section 5): a
mass-spring-damper ``m x'' + c x' + k x = u(t)`` driven by a piecewise-constant
random input, integrated with classical fourth-order Runge-Kutta; regressors
are lagged inputs and the target is the noisy position.  The paper's own data
set (DaRUS-4743) is not available here; this generator stands in for it with
the paper's shapes (N = M = 2^13, 8 or 128 regressors, powers of two).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> int:
    """Key of sub-stream ``stream`` of ``seed`` (first output of a SplitMix64 seeded by both)."""
    base = (int(seed) * 0x100000001B3 + int(stream) * 0x9E3779B1 + 0x632BE59BD9B4E019) & _MASK64
    return int(_mix(np.array([base], dtype=np.uint64))[0])


def splitmix64(key: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 sequence seeded with ``key``."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(key & _MASK64) + idx * _GOLDEN
    return _mix(state)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``count`` doubles uniform on [lo, hi) from sub-stream ``stream`` of ``seed``."""
    bits = splitmix64(stream_key(seed, stream), count)
    u = (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller from sub-stream ``stream`` of ``seed``."""
    half = (count + 1) // 2
    u = uniform(seed, stream, 2 * half)
    u1 = 1.0 - u[0::2]            # (0, 1]: keeps log finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * half)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def msd_simulate(u: np.ndarray, m, c, k, dt: float = 0.1) -> np.ndarray:
    """Positions x(t_j), j = 0..T-1, of ``m x'' + c x' + k x = u`` from rest.

    ``u`` has shape (T,) or (B, T) (a batch of systems, each with its own m, c,
    k given as arrays of shape (B,)).  ``u[..., j]`` is held constant over
    [j dt, (j+1) dt); x(t_0) = x'(t_0) = 0; classical RK4, one step per sample.
    """
    u = np.asarray(u, dtype=np.float64)
    batched = u.ndim == 2
    U = u if batched else u[None, :]
    B, T = U.shape
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), (B,))
    c = np.broadcast_to(np.asarray(c, dtype=np.float64), (B,))
    k = np.broadcast_to(np.asarray(k, dtype=np.float64), (B,))
    x = np.zeros(B)
    v = np.zeros(B)
    out = np.empty((B, T))
    for j in range(T):
        out[:, j] = x
        uj = U[:, j]

        def acc(xx, vv):
            return (uj - c * vv - k * xx) / m

        k1x, k1v = v, acc(x, v)
        k2x, k2v = v + 0.5 * dt * k1v, acc(x + 0.5 * dt * k1x, v + 0.5 * dt * k1v)
        k3x, k3v = v + 0.5 * dt * k2v, acc(x + 0.5 * dt * k2x, v + 0.5 * dt * k2v)
        k4x, k4v = v + dt * k3v, acc(x + dt * k3x, v + dt * k3v)
        x = x + (dt / 6.0) * (k1x + 2.0 * k2x + 2.0 * k3x + k4x)
        v = v + (dt / 6.0) * (k1v + 2.0 * k2v + 2.0 * k3v + k4v)
    return out if batched else out[0]


def lagged_regressors(u: np.ndarray, n_reg: int) -> np.ndarray:
    """Row j holds (u_{j-1}, ..., u_{j-n_reg}), with u_{i<0} = 0.  Shape (..., T, n_reg)."""
    u = np.asarray(u, dtype=np.float64)
    T = u.shape[-1]
    Z = np.zeros(u.shape[:-1] + (T, n_reg))
    for lag in range(1, n_reg + 1):
        Z[..., lag:, lag - 1] = u[..., : T - lag]
    return Z


def msd_dataset(n_train: int, n_test: int, n_reg: int, seed: int,
                m: float = 1.0, c: float = 0.5, k: float = 2.0,
                noise_std: float = 0.1, dt: float = 0.1):
    """Mass-spring-damper regression set: (X, y, Xs, ys).

    u_j ~ U[-1, 1) i.i.d. (stream 0), y_j = x(j dt) + noise_std * N(0,1)
    (stream 1).  Samples 0..n_train-1 train, the next n_test test.  X and Xs
    are row-major (rows = samples), float64, C-contiguous.
    """
    T = n_train + n_test
    u = uniform(seed, 0, T, -1.0, 1.0)
    x = msd_simulate(u, m, c, k, dt)
    y_all = x + noise_std * normal(seed, 1, T)
    Z = lagged_regressors(u, n_reg)
    X = np.ascontiguousarray(Z[:n_train])
    Xs = np.ascontiguousarray(Z[n_train:])
    return X, np.ascontiguousarray(y_all[:n_train]), Xs, np.ascontiguousarray(y_all[n_train:])


def msd_system_params(seed: int):
    """Random system for the learned-initialiser corpus: m~U[0.5,2], c~U[0.1,1], k~U[0.5,5], noise~U[0.01,0.3]."""
    p = uniform(seed, 7, 4)
    return (0.5 + 1.5 * p[0], 0.1 + 0.9 * p[1], 0.5 + 4.5 * p[2], 0.01 + 0.29 * p[3])


def msd_corpus(seeds, n_train: int, n_reg: int, dt: float = 0.1):
    """Batch of training sets, one per seed, each from its own random system.

    Returns X (B, n_train, n_reg), y (B, n_train) and the (B, 4) array of
    (m, c, k, noise_std).
    """
    seeds = list(seeds)
    B = len(seeds)
    prm = np.array([msd_system_params(s) for s in seeds])
    U = np.stack([uniform(s, 0, n_train, -1.0, 1.0) for s in seeds])
    x = msd_simulate(U, prm[:, 0], prm[:, 1], prm[:, 2], dt)
    E = np.stack([normal(s, 1, n_train) for s in seeds])
    y = x + prm[:, 3:4] * E
    X = lagged_regressors(U, n_reg)
    return np.ascontiguousarray(X), np.ascontiguousarray(y), prm


def rff_frequencies(count: int = 8, seed: int = 4242) -> np.ndarray:
    """Fixed random-Fourier-feature frequencies omega_q ~ N(0, 1) for the data summary."""
    return normal(seed, 3, count)


def random_points(n: int, d: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n x d uniform points (row-major), for edge-case and invariant tests."""
    return uniform(seed, 5, n * d, lo, hi).reshape(n, d)
