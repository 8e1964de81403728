"""Seeded synthetic inputs for the IterNCGP hot path.

This module only draws random numbers: it holds none of the method's arithmetic
(no kernel evaluation, no likelihood, no solver).  Both the CPU oracle (through the
tests and the bench) and the CUDA path receive the arrays made here, so the two sides
always see bit-identical inputs.  Every generator is a NumPy PCG64 stream seeded by the
caller.

Workloads (shapes and distributions follow the paper's experiments, Sec. 5 and App. C):

* ``blobs``      -- C isotropic Gaussian blobs (sigma = 1) with centres uniform in a box;
                    balanced labels.  Used for the small FP64 case (N = 500, D = 2, C = 3)
                    and for the batched problems.
* ``sparse_clusters`` -- a synthetic stand-in for the MNIST experiment (App. C.4):
                    N x 784 rows with about 19 % non-zero entries uniform in (0, 1],
                    grouped in 10 clusters, each cluster with its own support set.
* ``gmm3d``      -- the paper's own large-scale Gaussian-mixture generator (App. C.3):
                    per-class mean uniform in [-1, 1]^3 and covariance U diag(lambda) U^T
                    with U the eigenvectors of A A^T (A uniform in [0, 1]^{3x3}) and
                    lambda uniform in [0.001, 0.1].
* ``batch_problems`` -- 256 independent blob problems of uneven N, D, C, lengthscale.
* ``normal``     -- standard-normal right-hand sides S for the kernel product bench.
* ``poisson_study`` -- the Poisson-regression study (App. C): 100 points in [0, 1], a
                    log-rate drawn from an RBF GP (random Fourier features), Poisson counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blobs(n: int, d: int, c: int, seed: int, box: float = 3.0, sigma: float = 1.0,
          centres: np.ndarray | None = None):
    """Return (X float64 n x d, y int32 n, centres c x d).

    Labels are balanced: y_n = n mod c, then shuffled.  x_n = centre_{y_n} + sigma * N(0, I).
    If ``centres`` is given it is reused (test points from the same blobs)."""
    g = _rng(seed)
    if centres is None:
        centres = g.uniform(-box, box, size=(c, d))
    y = (np.arange(n) % c).astype(np.int32)
    g.shuffle(y)
    X = centres[y] + sigma * g.standard_normal((n, d))
    return X.astype(np.float64), y, centres


def blobs_train_test(n_train: int, n_test: int, d: int, c: int, seed: int):
    """Train set from ``seed``; test set from ``seed + 1`` with the same centres."""
    X, y, centres = blobs(n_train, d, c, seed)
    Xs, ys, _ = blobs(n_test, d, c, seed + 1, centres=centres)
    return X, y, Xs, ys


def sparse_clusters(n: int, seed: int, d: int = 784, n_clusters: int = 10,
                    density: float = 0.19, keep: float = 0.9):
    """Return (X float32 n x d, y int32 n): sparse non-negative rows in clusters.

    Each cluster owns a random support set of round(density * d) coordinates.  A row of
    cluster k keeps each support coordinate with probability ``keep`` and switches on
    each off-support coordinate with the probability that makes the expected non-zero
    fraction equal ``density``.  Non-zero values are uniform in (0, 1]; the rest are 0."""
    g = _rng(seed)
    n_sup = int(round(density * d))
    supports = np.zeros((n_clusters, d), dtype=bool)
    for k in range(n_clusters):
        supports[k, g.choice(d, size=n_sup, replace=False)] = True
    p_off = max(0.0, (density * d - keep * n_sup) / (d - n_sup))
    y = (np.arange(n) % n_clusters).astype(np.int32)
    g.shuffle(y)
    prob = np.where(supports[y], keep, p_off)
    mask = g.random((n, d)) < prob
    vals = 1.0 - g.random((n, d))          # uniform in (0, 1]
    X = np.where(mask, vals, 0.0).astype(np.float32)
    return X, y


def gmm3d(n_per_class: int, seed_model: int, seed_draw: int, c: int = 10):
    """Return (X float64 (c*n_per_class) x 3, y int32): the paper's 3-D Gaussian mixture."""
    gm = _rng(seed_model)
    means = gm.uniform(-1.0, 1.0, size=(c, 3))
    covs = []
    for _ in range(c):
        A = gm.uniform(0.0, 1.0, size=(3, 3))
        _, U = np.linalg.eigh(A @ A.T)
        lam = gm.uniform(0.001, 0.1, size=3)
        covs.append((U * lam) @ U.T)
    gd = _rng(seed_draw)
    X = np.concatenate([gd.multivariate_normal(means[k], covs[k], size=n_per_class)
                        for k in range(c)])
    y = np.repeat(np.arange(c, dtype=np.int32), n_per_class)
    perm = gd.permutation(len(y))
    return X[perm], y[perm]


def normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return _rng(seed).standard_normal(shape).astype(dtype)


@dataclass
class BatchProblem:
    X: np.ndarray          # n x d float32
    y: np.ndarray          # n int32
    c: int
    lengthscale: float
    Xs: np.ndarray         # test points (n_test x d float32)


def batch_problems(count: int = 256, seed: int = 4, n_lo: int = 200, n_hi: int = 20000,
                   dims=(8, 16, 32, 64), c_lo: int = 2, c_hi: int = 10,
                   ell_lo: float = 0.3, ell_hi: float = 3.0, n_test: int = 64,
                   ell_per_sqrt_d: bool = False):
    """Independent blob problems of uneven size (batched-fit workload).

    N = floor(exp U[ln n_lo, ln n_hi]); D uniform over ``dims``; C uniform in
    {c_lo..c_hi}; RBF lengthscale exp U[ln ell_lo, ln ell_hi], times sqrt(D) when
    ``ell_per_sqrt_d`` (the kernel then sees distances on the scale of the blob spread)."""
    g = _rng(seed)
    out = []
    for i in range(count):
        n = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.choice(dims))
        c = int(g.integers(c_lo, c_hi + 1))
        ell = float(math.exp(g.uniform(math.log(ell_lo), math.log(ell_hi))))
        if ell_per_sqrt_d:
            ell *= math.sqrt(d)
        sub = int(g.integers(0, 2**31 - 1))
        X, y, centres = blobs(n, d, c, sub)
        Xs, _, _ = blobs(n_test, d, c, sub + 1, centres=centres)
        out.append(BatchProblem(X.astype(np.float32), y, c, ell, Xs.astype(np.float32)))
    return out


def one_latent(kind: str, n: int, seed: int, d: int = 2, n_test: int = 100):
    """Single-latent problems: X ~ U[-3, 3]^d, latent g(x) = sin(x_1) + x_2 / 2, and
    y ~ Bernoulli(1 / (1 + e^(-2 g))) ("bernoulli"), y ~ Poisson(e^g) ("poisson") or
    y = g + N(0, 0.1^2) ("gaussian").  Returns X, y, Xs (float32, labels int32)."""
    g = _rng(seed)
    X = g.uniform(-3.0, 3.0, size=(n + n_test, d))
    lat = np.sin(X[:, 0]) + (0.5 * X[:, 1] if d > 1 else 0.0)
    if kind == "bernoulli":
        y = (g.random(n + n_test) < 1.0 / (1.0 + np.exp(-2.0 * lat))).astype(np.int32)
    elif kind == "poisson":
        y = g.poisson(np.exp(lat)).astype(np.int32)
    else:
        y = (lat + 0.1 * g.standard_normal(n + n_test)).astype(np.float32)
    X = X.astype(np.float32)
    return X[:n], y[:n], X[n:]


def poisson_study(seed: int, runs: int = 10, n: int = 100, lengthscale: float = 0.1,
                  outputscale: float = 5.0, features: int = 4096):
    """The Poisson-regression study's data (App. C): n inputs linearly spaced in [0, 1]; one
    fixed log-rate function f drawn from a zero-mean GP with an RBF covariance of the given
    lengthscale and outputscale; `runs` training count vectors y_r ~ Poisson(e^f(x)) at
    those inputs, plus `runs` test count vectors drawn the same way.

    The GP draw is a random-Fourier-feature sample, f(x) = sqrt(2 s / M) sum_m
    w_m cos(omega_m x + b_m) with omega_m ~ N(0, 1 / l^2), b_m ~ U[0, 2 pi), w_m ~ N(0, 1)
    and M = `features`: a sample whose covariance tends to s exp(-(x - x')^2 / (2 l^2))
    as M grows, made of random numbers only.  Returns X (n x 1 float32), f (n, float64),
    Y (runs x n int32), Y_test (runs x n int32)."""
    g = _rng(seed)
    x = np.linspace(0.0, 1.0, n)
    om = g.standard_normal(features) / lengthscale
    b = g.uniform(0.0, 2.0 * math.pi, size=features)
    w = g.standard_normal(features)
    f = math.sqrt(2.0 * outputscale / features) * (np.cos(np.outer(x, om) + b) @ w)
    lam = np.exp(f)
    Y = g.poisson(lam, size=(runs, n)).astype(np.int32)
    Yt = g.poisson(lam, size=(runs, n)).astype(np.int32)
    return x.reshape(n, 1).astype(np.float32), f, Y, Yt


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of ``rate`` per second."""
    g = _rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(out)
        out.append(t)


# ---- named workloads ---------------------------------------------------------------

def workload_small(n_train: int = 500, n_test: int = 200, seed: int = 0):
    """Small multi-class case: 3 blobs in 2-D, centres uniform in [-3, 3]^2."""
    return blobs_train_test(n_train, n_test, d=2, c=3, seed=seed)


def workload_kernel_bench(n: int = 60000, p: int = 80, seed: int = 2, n_test: int = 10000):
    """Large kernel-product workload: 784-D sparse clusters, S ~ N(0, 1) of n x p."""
    X, y = sparse_clusters(n + n_test, seed)
    S = normal((n, p), seed + 100)
    return X[:n], y[:n], X[n:], y[n:], S
