"""Failure detection without a GPU fault: a bounded wait that runs out on the device is
reported as ITERGP_ETIMEOUT through the status word, and the context stays usable."""
import time

import numpy as np
import pytest
import torch

import oracle.itergp_oracle as O
from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_a_wait_that_runs_out_is_reported_and_the_context_stays_usable(native):
    assert native.sync_status() == native.OK
    t0 = time.time()
    native.selftest_wait(limit_ns=20_000_000)          # 20 ms, nothing ever arrives
    assert native.sync_status() == native.ETIMEOUT
    assert time.time() - t0 < 10.0
    assert native.sync_status() == native.OK           # read and cleared
    X = datagen.normal((300, 5), 1)
    S = datagen.normal((300, 3), 2)
    tX, tS = torch.as_tensor(X, device=DEV), torch.as_tensor(S, device=DEV)
    ref = O.kmatvec(X, X, S, O.Kernel(O.RBF, 2.0, 1.0))
    for prec in ("fp32", "bf16x3"):
        Y = native.kmatvec(tX, tX, tS, kind="rbf", lengthscale=2.0, precision=prec)
        assert np.linalg.norm(Y.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
    assert native.sync_status() == native.OK


def test_selftest_limits_are_validated(native):
    with pytest.raises(native.ItergpError):
        native.selftest_wait(limit_ns=10)
    with pytest.raises(native.ItergpError):
        native.selftest_wait(limit_ns=10_000_000_000)
