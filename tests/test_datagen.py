"""The seeded input generators follow the recipes the workloads are stated with: shapes,
value ranges, label balance, sparsity and the distributions of the batched problems.
Each generator is deterministic in its seed (both sides of every parity test and the
bench see bit-identical arrays)."""
import math

import numpy as np

from paper_2310_20285_gb300 import datagen


def test_generators_are_deterministic_in_their_seed():
    a = datagen.sparse_clusters(300, seed=5)
    b = datagen.sparse_clusters(300, seed=5)
    c = datagen.sparse_clusters(300, seed=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    g1, g2 = datagen.gmm3d(50, 1, 2), datagen.gmm3d(50, 1, 2)
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])
    p1 = datagen.batch_problems(count=4, seed=4, n_hi=500)
    p2 = datagen.batch_problems(count=4, seed=4, n_hi=500)
    assert all(np.array_equal(x.X, y.X) and x.lengthscale == y.lengthscale for x, y in zip(p1, p2))


def test_blobs_are_balanced_around_their_centres():
    X, y, centres = datagen.blobs(3000, 2, 3, seed=0)
    assert X.shape == (3000, 2) and y.dtype == np.int32
    assert np.bincount(y).tolist() == [1000, 1000, 1000]
    assert np.all(np.abs(centres) <= 3.0)
    for k in range(3):                     # unit-variance blobs around their centres
        Z = X[y == k] - centres[k]
        assert np.allclose(Z.mean(0), 0.0, atol=0.1)
        assert np.allclose(Z.std(0), 1.0, atol=0.08)
    # test points share the training centres
    Xt, yt, Xs, ys = datagen.blobs_train_test(600, 300, d=2, c=3, seed=0)
    for k in range(3):
        assert np.linalg.norm(Xt[yt == k].mean(0) - Xs[ys == k].mean(0)) < 0.35


def test_sparse_clusters_match_the_kernel_bench_recipe():
    X, y = datagen.sparse_clusters(4000, seed=2)
    assert X.shape == (4000, 784) and X.dtype == np.float32
    nz = X != 0
    assert abs(nz.mean() - 0.19) < 0.005                 # expected non-zero fraction
    assert X.min() >= 0.0 and X.max() <= 1.0 and np.all(X[nz] > 0)
    assert np.bincount(y).tolist() == [400] * 10
    # each cluster has a common support: its coordinates on in about 90 % of its rows
    for k in range(10):
        on = nz[y == k].mean(0)
        support = on > 0.5
        assert support.sum() == round(0.19 * 784)
        assert abs(on[support].mean() - 0.9) < 0.02
    vals = X[nz]                                         # non-zeros uniform in (0, 1]
    assert abs(vals.mean() - 0.5) < 0.01 and abs(vals.var() - 1 / 12) < 0.005


def test_gmm3d_follows_the_paper_generator():
    X, y = datagen.gmm3d(4000, seed_model=1, seed_draw=2)
    assert X.shape == (40000, 3) and np.bincount(y).tolist() == [4000] * 10
    for k in range(10):
        Z = X[y == k]
        assert np.all(np.abs(Z.mean(0)) <= 1.0 + 0.02)   # means uniform in [-1, 1]^3
        ev = np.linalg.eigvalsh(np.cov(Z.T))             # covariance eigenvalues in [0.001, 0.1]
        assert ev.min() > 0.0008 and ev.max() < 0.11


def test_batch_problems_span_the_stated_ranges():
    probs = datagen.batch_problems(count=256, seed=4)
    ns = np.array([p.X.shape[0] for p in probs])
    ds = {p.X.shape[1] for p in probs}
    cs = np.array([p.c for p in probs])
    ells = np.array([p.lengthscale for p in probs])
    assert ns.min() >= 200 and ns.max() < 20000
    assert abs(np.log(ns).mean() - (math.log(200) + math.log(20000)) / 2) < 0.4   # log-uniform
    assert ds == {8, 16, 32, 64}
    assert cs.min() == 2 and cs.max() == 10
    assert ells.min() >= 0.3 and ells.max() <= 3.0
    assert all(np.bincount(p.y, minlength=p.c).max() - np.bincount(p.y, minlength=p.c).min() <= 1
               for p in probs)                            # balanced labels
    assert sum(ns) == 1254572                             # the batched workload's total N


def test_one_latent_labels_follow_their_likelihoods():
    X, y, Xs = datagen.one_latent("poisson", 20000, seed=1, n_test=10)
    lat = np.sin(X[:, 0].astype(np.float64)) + 0.5 * X[:, 1]
    assert X.shape == (20000, 2) and Xs.shape == (10, 2) and np.all(np.abs(X) <= 3.0)
    assert y.min() >= 0 and abs(y.mean() - np.exp(lat).mean()) < 0.05
    _, yb, _ = datagen.one_latent("bernoulli", 20000, seed=1, n_test=10)
    assert set(np.unique(yb).tolist()) == {0, 1}
    assert abs(yb.mean() - (1 / (1 + np.exp(-2 * lat))).mean()) < 0.02
    _, yg, _ = datagen.one_latent("gaussian", 20000, seed=1, n_test=10)
    assert yg.dtype == np.float32 and abs((yg - lat).std() - 0.1) < 0.005


def test_poisson_arrivals_have_the_stated_rate():
    t = datagen.poisson_arrivals(2000.0, 5.0, seed=5)
    assert np.all(np.diff(t) > 0) and t.max() < 5.0
    assert abs(len(t) / 5.0 - 2000.0) < 3 * math.sqrt(2000.0 * 5.0) / 5.0
