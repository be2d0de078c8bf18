"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and describes problem data only; it holds
none of the method's arithmetic and imports neither the oracle nor the CUDA
package.  Vectors are FP64 numpy arrays in the compact interior numbering
(interior nodes of the level, lexicographic, dimension 0 fastest).

The workloads follow the shapes of the paper's experiments (Poisson on the
unit square/cube with Q_k elements, Section 2 and Section 4.2): random
residual vectors, random right-hand sides, manufactured sine solutions and a
stream of solve requests.
"""

import math

import numpy as np


def n_interior(d, k, level):
    """Number of interior DoFs of Q_k on 2^level cells per direction."""
    return (k * 2 ** level - 1) ** d


def normal_vector(n, seed):
    """N(0, 1) vector of length n (seeded numpy PCG64)."""
    return np.random.default_rng(seed).standard_normal(n)


def uniform_vector(n, seed, lo=-1.0, hi=1.0):
    """U[lo, hi) vector of length n (seeded numpy PCG64)."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def sine_modes(d, seed, n_modes=4, qmax=4):
    """Coefficients a_m ~ U[-1,1] and integer frequencies q_{m,t} ~ U{1..qmax}.

    They describe f(x) = sum_m a_m prod_t sin(pi q_{m,t} x_t).
    Returns (coef (n_modes,), freq (n_modes, d) int32).
    """
    rng = np.random.default_rng(seed)
    coef = rng.uniform(-1.0, 1.0, n_modes)
    freq = rng.integers(1, qmax + 1, size=(n_modes, d)).astype(np.int32)
    return coef, freq


def manufactured_sine(d):
    """u = prod sin(pi x_t), f = d pi^2 u, as one sine mode: (coef, freq)."""
    return np.array([d * math.pi ** 2]), np.ones((1, d), dtype=np.int32)


def sine_function(coef, freq):
    """Callable f(X) for X of shape (npts, d) from (coef, freq)."""
    coef = np.asarray(coef, dtype=np.float64)
    freq = np.asarray(freq)

    def f(X):
        out = np.zeros(len(X))
        for a, q in zip(coef, freq):
            out += a * np.prod(np.sin(math.pi * q[None, :] * X), axis=1)
        return out
    return f


def exact_sine_solution(d):
    """u(X) = prod sin(pi x_t) for X of shape (npts, d)."""
    return lambda X: np.prod(np.sin(math.pi * X), axis=1)


def request_stream(n_requests, rate_per_s, seed, dofs_range=(1e4, 2e7),
                   dims=(2, 3), degrees=(2, 3, 4, 5, 6)):
    """Poisson-arrival stream of Poisson-solve requests.

    Each request draws d and k uniformly, then a level uniformly among the
    levels whose interior DoF count lies in ``dofs_range``, and four sine
    modes for its right-hand side.  Returns a list of dicts with keys
    t_arrival (s), d, k, level, coef, freq, seed.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        d = int(rng.choice(dims))
        k = int(rng.choice(degrees))
        levels = [l for l in range(1, 16)
                  if dofs_range[0] <= n_interior(d, k, l) <= dofs_range[1]]
        level = int(rng.choice(levels))
        coef, freq = sine_modes(d, seed=int(rng.integers(0, 2 ** 31)))
        out.append(dict(t_arrival=t, d=d, k=k, level=level, coef=coef, freq=freq, index=i))
    return out
