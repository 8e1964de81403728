"""Parity of the CUDA kernel product Y = k(A, B) S (App. B.3.1) against the FP64 oracle.

Bars: FP32 paths (fp32, bf16x3) -- normwise relative error <= 1e-4 and componentwise
|Y - Y_ref| <= 1e-4 (|K| |S|) + tiny; BF16 and TF32 paths -- normwise <= 1e-2 (their
gated quantity is the predictive mean; the product's error is recorded here).  The TF32
path also meets the FP32 bar against the product of its TF32-rounded inputs."""
import math

import numpy as np
import pytest
import torch

import oracle.itergp_oracle as O
from numerics import round_tf32
from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.gpu

FP32_PATHS = ["fp32", "bf16x3"]
ALL_PATHS = ["fp32", "bf16x3", "bf16_comp", "bf16", "tf32"]
KINDS = {"rbf": O.RBF, "matern32": O.MATERN32}


def run(native, A, B, S, kind, ell, s, prec):
    dev = torch.device("cuda:0")
    tA = torch.as_tensor(A, dtype=torch.float32, device=dev).contiguous()
    tB = tA if B is A else torch.as_tensor(B, dtype=torch.float32, device=dev).contiguous()
    tS = torch.as_tensor(S, dtype=torch.float32, device=dev).contiguous()
    Y = native.kmatvec(tA, tB, tS, kind=kind, lengthscale=ell, outputscale=s, precision=prec)
    assert native.sync_status() == 0
    return Y.cpu().numpy().astype(np.float64)


def check(Y, A, B, S, kind, ell, s, prec, norm_tol=None):
    # the oracle sees the same FP32 inputs the GPU saw
    A64, B64, S64 = (np.asarray(x, dtype=np.float32).astype(np.float64) for x in (A, B, S))
    kern = O.Kernel(KINDS[kind], ell, s)
    K = O.kernel_matrix(A64, B64, kern)
    ref = K @ S64
    scale = np.abs(K) @ np.abs(S64)
    err = np.abs(Y - ref)
    rel = np.linalg.norm(Y - ref) / max(np.linalg.norm(ref), 1e-300)
    if prec in FP32_PATHS:
        assert rel <= 1e-4, (prec, rel)
        assert np.all(err <= 1e-4 * scale + 1e-30), (prec, float((err / (scale + 1e-30)).max()))
    else:
        assert rel <= (norm_tol or 1e-2), (prec, rel)
    return rel


@pytest.mark.parametrize("prec", ALL_PATHS)
@pytest.mark.parametrize("kind", ["rbf", "matern32"])
def test_ragged_multi_tile(native, prec, kind):
    g = np.random.default_rng(11)
    m, n, d, p = 300, 517, 70, 21          # 3 row tiles, 5 column chunks, 2 D slices, ragged
    A = g.standard_normal((m, d)).astype(np.float32)
    B = g.standard_normal((n, d)).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    ell = math.sqrt(d)
    Y = run(native, A, B, S, kind, ell, 0.7, prec)
    check(Y, A, B, S, kind, ell, 0.7, prec)


@pytest.mark.parametrize("prec", ALL_PATHS)
def test_symmetric_product_small_workload(native, prec):
    """K(X, X) S on the small 2-D blob workload, RBF l = 1 (distance cancellation matters)."""
    X, y, _, _ = datagen.workload_small()
    S = datagen.normal((X.shape[0], 3), 5)
    tX = X.astype(np.float32)
    Y = run(native, tX, tX, S, "rbf", 1.0, 1.0, prec)
    check(Y, tX, tX, S, "rbf", 1.0, 1.0, prec, norm_tol=2e-2)


@pytest.mark.parametrize("prec", ALL_PATHS)
def test_many_output_columns_span_several_p_tiles(native, prec):
    g = np.random.default_rng(5)
    m, n, d, p = 200, 390, 33, 290          # p > 256 -> several P tiles on every path
    A = g.uniform(-1, 1, (m, d)).astype(np.float32)
    B = g.uniform(-1, 1, (n, d)).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    ell = math.sqrt(d)
    Y = run(native, A, B, S, "matern32", ell, 1.2, prec)
    check(Y, A, B, S, "matern32", ell, 1.2, prec)


@pytest.mark.parametrize("prec", ALL_PATHS)
def test_high_dimension_sparse_rows(native, prec):
    """784-D sparse cluster rows (the kernel-bench distribution), Matern l = sqrt(D)."""
    X, _ = datagen.sparse_clusters(700, seed=2)
    S = datagen.normal((700, 80), 102)
    Y = run(native, X, X, S, "matern32", 28.0, 1.0, prec)
    check(Y, X, X, S, "matern32", 28.0, 1.0, prec)


@pytest.mark.parametrize("prec", ALL_PATHS)
@pytest.mark.parametrize("m,n,d,p", [(1, 1, 1, 1), (1, 300, 3, 2), (129, 1, 5, 17), (5, 128, 64, 16),
                                     (128, 256, 128, 128), (7, 9, 200, 1)])
def test_edge_shapes(native, prec, m, n, d, p):
    g = np.random.default_rng(m * 1000 + n)
    A = g.standard_normal((m, d)).astype(np.float32)
    B = g.standard_normal((n, d)).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    ell = math.sqrt(d) + 0.5
    Y = run(native, A, B, S, "rbf", ell, 1.0, prec)
    check(Y, A, B, S, "rbf", ell, 1.0, prec, norm_tol=2e-2)


@pytest.mark.parametrize("prec", ALL_PATHS)
def test_empty_inputs(native, prec):
    dev = torch.device("cuda:0")
    A = torch.randn(5, 3, device=dev)
    B = torch.empty(0, 3, device=dev)
    S = torch.empty(0, 4, device=dev)
    Y = torch.full((5, 4), 7.0, device=dev)
    native.kmatvec(A, B, S, precision=prec, out=Y)
    torch.cuda.synchronize()
    assert torch.all(Y == 0)
    Y0 = native.kmatvec(torch.empty(0, 3, device=dev), A, torch.randn(5, 2, device=dev), precision=prec)
    assert Y0.shape == (0, 2)


@pytest.mark.parametrize("kind,d", [("rbf", 2), ("matern32", 70), ("matern32", 784)])
def test_tf32_path_is_exact_on_tf32_rounded_inputs(native, kind, d):
    """The TF32 form rounds each coordinate once to 10 mantissa bits and otherwise computes
    like BF16X3 (norms of the rounded rows, FP32 accumulation, split weights), so against
    the FP64 product of the rounded inputs it meets the FP32 bar."""
    g = np.random.default_rng(d)
    m, n, p = 300, 517, 21
    A = (g.standard_normal((m, d)) * 2).astype(np.float32)
    B = (g.standard_normal((n, d)) * 2).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    ell = 1.0 if d == 2 else math.sqrt(d)
    Y = run(native, A, B, S, kind, ell, 1.0, "tf32")
    check(Y, round_tf32(A), round_tf32(B), S, kind, ell, 1.0, "fp32")


def test_paths_agree_and_are_deterministic(native):
    g = np.random.default_rng(3)
    A = torch.as_tensor(g.standard_normal((260, 40)), dtype=torch.float32, device="cuda")
    S = torch.as_tensor(g.standard_normal((260, 9)), dtype=torch.float32, device="cuda")
    y1 = native.kmatvec(A, A, S, precision="bf16x3", lengthscale=4.0)
    y2 = native.kmatvec(A, A, S, precision="bf16x3", lengthscale=4.0)
    y3 = native.kmatvec(A, A, S, precision="fp32", lengthscale=4.0)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    assert torch.linalg.norm(y1 - y3) / torch.linalg.norm(y3) < 1e-4


@pytest.mark.parametrize("prec", ["bf16x3", "fp32", "tf32"])
def test_full_size_kernel_bench_sampled_rows(native, prec):
    """N = 60000, D = 784, P = 80, Matern-3/2 l = 28 -- the kernel-bench workload in the
    launch configuration the bench times; 48 sampled output rows against the oracle."""
    X, _, _, _, S = datagen.workload_kernel_bench()
    dev = torch.device("cuda:0")
    tX = torch.as_tensor(X, device=dev)
    tS = torch.as_tensor(S, device=dev)
    Y = native.kmatvec(tX, tX, tS, kind="matern32", lengthscale=28.0, outputscale=1.0, precision=prec)
    assert native.sync_status() == 0
    rows = np.random.default_rng(0).choice(X.shape[0], 48, replace=False)
    rows = np.concatenate([rows, [0, X.shape[0] - 1]])
    Ys = Y[torch.as_tensor(rows, device=dev)].cpu().numpy().astype(np.float64)
    check(Ys, X[rows], X, S, "matern32", 28.0, 1.0, prec)
