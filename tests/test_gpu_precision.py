"""Precision forms against the FP64 oracle on 5000-point inputs: the small blob workload's
generator drawn at N = 5000 (D = 2, C = 3, RBF l = 1) and the first 5000 rows of the
784-D kernel-bench data (Matern-3/2, l = 28).  Reports the relative error of K.S, of every
Newton iterate f_i and of the predictive mean per precision (written to
$ITERGP_REPORT_DIR/precision_report.json when that variable is set) and gates each
against its stated bound."""
import json
import os

import numpy as np
import pytest
import torch

import oracle.itergp_oracle as O
from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
PRECS = ["fp32", "bf16x3", "bf16_comp", "bf16", "tf32"]
REPORT = {}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16x3_bound(X, ell):
    """BF16X3 (FP16 hi/lo rows with tile scales, BF16 hi/lo weights) is held to the FP32
    bar."""
    return 1e-4


def write_report():
    d = os.environ.get("ITERGP_REPORT_DIR")
    if d:
        with open(os.path.join(d, "precision_report.json"), "w") as f:
            json.dump(REPORT, f, indent=1)


@pytest.mark.parametrize("data", ["blobs5000", "kernel_bench5000"])
def test_kernel_product_errors(native, data):
    if data == "blobs5000":
        X, y, Xs, ys = datagen.blobs_train_test(5000, 200, d=2, c=3, seed=0)
        kern, kind = O.Kernel(O.RBF, 1.0, 1.0), "rbf"
    else:
        X, y, Xs, ys, _ = datagen.workload_kernel_bench(n=5000, n_test=10)
        kern, kind = O.Kernel(O.MATERN32, 28.0, 1.0), "matern32"
    X = np.asarray(X, dtype=np.float32)
    S = datagen.normal((5000, 24), 77)
    ref = O.kmatvec(X.astype(np.float64), X.astype(np.float64), S.astype(np.float64), kern)
    tX, tS = torch.as_tensor(X, device=DEV), torch.as_tensor(S, device=DEV)
    errs = {}
    for prec in PRECS:
        Y = native.kmatvec(tX, tX, tS, kind=kind, lengthscale=kern.lengthscale, precision=prec)
        errs[prec] = rel(Y.cpu(), ref)
    REPORT[f"K.S {data}"] = errs
    write_report()
    assert errs["fp32"] <= 1e-5
    assert errs["bf16x3"] <= 1e-4
    assert errs["bf16_comp"] <= 1e-2 and errs["bf16"] <= 2e-2 and errs["tf32"] <= 1e-2


def test_newton_iterates_and_predictive_mean(native):
    """10 Newton steps x <= 50 CG iterations, R = 50, tolerances 1e-5 (the small workload's
    schedule) at N = 5000; f_i from fits stopped after i steps."""
    X, y, Xs, ys = datagen.blobs_train_test(5000, 200, d=2, c=3, seed=0)
    X = X.astype(np.float32)
    kern = O.Kernel(O.RBF, 1.0, 1.0)
    X64 = X.astype(np.float64)
    ref = O.iterncgp_fit(X64, O.Softmax(y, 3), 3, kern, max_newton=10, max_iters=50, R=50)
    em, _, _ = O.predict(Xs.astype(np.float32).astype(np.float64), X64, ref.v, ref.Q, kern, 3)
    tX, ty = torch.as_tensor(X, device=DEV), torch.as_tensor(y, device=DEV)
    tXs = torch.as_tensor(Xs.astype(np.float32), device=DEV)
    out = {}
    for prec in PRECS:
        fi = []
        for i in range(1, 11):
            m = native.fit(tX, ty, 3, kind="rbf", lengthscale=1.0, precision=prec, max_newton=i,
                           max_iters=50, rank=50)
            fi.append(rel(m.arrays()["f"].cpu(), ref.fs[i]))
            if i == 10:
                mean, _, _ = m.predict(tXs)
                mean_err = rel(mean.cpu(), em)
            m.free()
        out[prec] = {"f_i": fi, "mean": mean_err}
    REPORT["fit blobs5000 (10 x 50, R=50)"] = out
    write_report()
    assert max(out["fp32"]["f_i"]) <= 1e-4 and out["fp32"]["mean"] <= 1e-4
    b = bf16x3_bound(X, 1.0)
    assert out["bf16x3"]["mean"] <= b
    for prec in ("bf16_comp", "bf16", "tf32"):
        assert out[prec]["mean"] <= 1e-2, (prec, out[prec])
