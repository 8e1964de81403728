"""One kernel per output GP (the C latent GPs are independent, Sec. 5 / App. C.3, here
each with its own hyperparameters): the grouped product, the fit (Alg. 1-3) and the
predictive (Eqs. 9-10) against the FP64 oracle.

Bars as for the shared kernel: FP32 paths (fp32, bf16x3) within 1e-4 normwise on
products, f, v and the predictive mean, 1e-4 absolute on probabilities and 1e-3 s on
variances; BF16X3 where the split's bound 2^-15 max|x|^2 / l_min^2 exceeds 1e-4, that
bound."""
import numpy as np
import pytest
import torch

import oracle.itergp_oracle as O
from numerics import round_tf32
from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
KIND = {"rbf": O.RBF, "matern32": O.MATERN32}
KERNS3 = [("rbf", 1.0, 1.3), ("matern32", 1.4, 0.6), ("rbf", 2.0, 1.0)]


def t32(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device=DEV)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def okerns(ks):
    return O.ClassKernels(tuple(O.Kernel(KIND[k], ell, s) for k, ell, s in ks))


def split_tol(prec, X, ks):
    """FP32 and BF16X3 (FP16 hi/lo rows, 22 significant bits) are held to the same 1e-4."""
    return 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,p", [(700, 700, 6), (300, 1041, 7), (129, 260, 3), (1000, 513, 10)])
def test_grouped_product_matches_the_oracle(native, prec, m, n, p):
    """Column j uses class j mod 3's kernel; ragged tiles, uneven column counts per class."""
    g = np.random.default_rng(m + n + p)
    A = g.standard_normal((m, 5)).astype(np.float32)
    B = A if m == n else g.standard_normal((n, 5)).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    tA = t32(A)
    tB = tA if B is A else t32(B)
    Y = native.kmatvec_classes(tA, tB, t32(S), KERNS3, precision=prec).cpu().numpy()
    assert native.sync_status() == 0
    ref = O.kmatvec_classes(A.astype(np.float64), B.astype(np.float64), S.astype(np.float64), okerns(KERNS3), 3)
    assert rel(Y, ref) <= split_tol(prec, np.vstack([A, B]), KERNS3), rel(Y, ref)


@pytest.mark.parametrize("m,n,p", [(700, 700, 6), (300, 1041, 7)])
def test_grouped_tf32_product_is_exact_on_tf32_rounded_inputs(native, m, n, p):
    """The TF32 form with one kernel per class: against the FP64 grouped product of the
    TF32-rounded inputs it meets the FP32 bar."""
    g = np.random.default_rng(m + n + p + 1)
    A = g.standard_normal((m, 5)).astype(np.float32)
    B = A if m == n else g.standard_normal((n, 5)).astype(np.float32)
    S = g.standard_normal((n, p)).astype(np.float32)
    tA = t32(A)
    tB = tA if B is A else t32(B)
    Y = native.kmatvec_classes(tA, tB, t32(S), KERNS3, precision="tf32").cpu().numpy()
    assert native.sync_status() == 0
    Ar, Br = round_tf32(A).astype(np.float64), round_tf32(B).astype(np.float64)
    ref = O.kmatvec_classes(Ar, Br, S.astype(np.float64), okerns(KERNS3), 3)
    assert rel(Y, ref) <= 1e-4, rel(Y, ref)


def test_equal_class_kernels_reduce_to_the_shared_product(native):
    g = np.random.default_rng(4)
    A = t32(g.standard_normal((640, 6)))
    S = t32(g.standard_normal((640, 8)))
    same = [("matern32", 1.5, 0.8)] * 4
    Y1 = native.kmatvec_classes(A, A, S, same, precision="fp32").cpu().numpy()
    Y2 = native.kmatvec(A, A, S, kind="matern32", lengthscale=1.5, outputscale=0.8, precision="fp32").cpu().numpy()
    assert rel(Y1, Y2) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_fit_and_predict_with_class_kernels_match_the_oracle(native, prec):
    """Softmax, residual (CG) actions, 4 Newton steps x 10 iterations, R = 20."""
    X, y, Xs, _ = datagen.workload_small(n_train=400, n_test=80)
    X32, Xs32 = X.astype(np.float32), Xs.astype(np.float32)
    kerns = okerns(KERNS3)
    ref = O.iterncgp_fit(X32.astype(np.float64), O.Softmax(y, 3), 3, kerns, max_newton=4, max_iters=10, R=20,
                         tol_abs=0, tol_rel=0)
    m = native.fit(t32(X32), torch.as_tensor(y, dtype=torch.int32, device=DEV), 3, class_kernels=KERNS3,
                   precision=prec, max_newton=4, max_iters=10, rank=20, tol_abs=0.0, tol_rel=0.0)
    tol = split_tol(prec, X32, KERNS3)
    assert m.report.newton_steps == 4
    assert [m.report.iters[i] for i in range(4)] == [inf.iters for inf in ref.infos]
    arr = m.arrays()
    assert rel(arr["f"].cpu(), ref.f) <= tol
    assert rel(arr["v"].cpu(), ref.v) <= tol
    for i in range(4):
        assert abs(m.report.objective[i] - ref.objectives[i]) <= tol * abs(ref.objectives[i])
    mean, var, probs = m.predict(t32(Xs32))
    em, ev, ep = O.predict(Xs32.astype(np.float64), X32.astype(np.float64), ref.v, ref.Q, kerns, 3)
    assert rel(mean.cpu(), em) <= tol
    assert np.max(np.abs(var.cpu().numpy() - ev)) <= 1e-3 * max(k[2] for k in KERNS3)
    assert np.max(np.abs(probs.cpu().numpy() - ep)) <= 10 * tol
    m.free()


def test_unit_actions_with_class_kernels_reach_the_exact_step(native):
    """NC unit-vector actions solve the pseudo-target system exactly: f_1 is the oracle's
    direct solve under the per-class prior."""
    X, y, _ = datagen.blobs(40, 2, 3, 5)
    X32 = X.astype(np.float32)
    kerns = okerns(KERNS3)
    m = native.fit(t32(X32), torch.as_tensor(y, dtype=torch.int32, device=DEV), 3, class_kernels=KERNS3,
                   precision="fp32", policy="unit", max_newton=1, max_iters=120, rank=-1, tol_abs=0.0,
                   tol_rel=0.0)
    _, f1 = O.exact_newton_step(X32.astype(np.float64), O.Softmax(y, 3), np.zeros((40, 3)), np.zeros((40, 3)), kerns)
    assert rel(m.arrays()["f"].cpu(), f1) <= 1e-3
    m.free()


def test_gaussian_likelihood_with_class_kernels(native):
    """Independent GP regression per output (W^-1 = noise I): against the oracle's fit."""
    g = np.random.default_rng(12)
    X = g.uniform(-2, 2, (300, 2)).astype(np.float32)
    Yr = np.stack([np.sin(2 * X[:, 0]), np.cos(X[:, 1]), X[:, 0] * X[:, 1]], axis=1)
    Yr = (Yr + 0.1 * g.standard_normal(Yr.shape)).astype(np.float32)
    kerns = okerns(KERNS3)
    ref = O.iterncgp_fit(X.astype(np.float64), O.Gaussian(Yr.astype(np.float64), 0.25), 3, kerns, max_newton=2,
                         max_iters=15, R=30, tol_abs=0, tol_rel=0)
    m = native.fit(t32(X), t32(Yr), 3, class_kernels=KERNS3, precision="fp32", likelihood="gaussian",
                   noise=0.25, max_newton=2, max_iters=15, rank=30, tol_abs=0.0, tol_rel=0.0)
    assert rel(m.arrays()["f"].cpu(), ref.f) <= 1e-3
    m.free()


def test_batched_call_with_class_kernels_equals_single_fits(native):
    probs = datagen.batch_problems(count=3, seed=21, n_lo=200, n_hi=500, dims=(4,), c_lo=3, c_hi=3,
                                   ell_lo=1.0, ell_hi=2.0, n_test=10, ell_per_sqrt_d=True)
    sched = dict(max_newton=2, max_iters=5, rank=10, tol_abs=0.0, tol_rel=0.0)
    ks = [KERNS3, list(reversed(KERNS3)), KERNS3[:1] * 3]
    dev = [(t32(p.X), torch.as_tensor(p.y, device=DEV), p.c, p.lengthscale, 1.0, k) for p, k in zip(probs, ks)]
    batch = native.fit_batch(dev, precision="bf16x3", **sched)
    for (X, y, c, _, _, k), mb in zip(dev, batch):
        ms = native.fit(X, y, c, class_kernels=k, precision="bf16x3", **sched)
        assert torch.equal(mb.arrays()["f"], ms.arrays()["f"])
        ms.free()
        mb.free()
