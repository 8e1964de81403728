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


def test_fit_wait_limit_and_peak_bytes_reach_the_report(native):
    """A fit with its own device-wait bound (wait_limit_ns, here 0.5 s, far above what
    any wait of this small fit takes) completes normally, and its report carries the
    call's peak pool bytes: at least the model it keeps, at most what the device has."""
    X, y, _ = datagen.blobs(700, 2, 3, 9)
    m = native.fit(torch.as_tensor(X.astype(np.float32), device=DEV), torch.as_tensor(y, device=DEV), 3,
                   precision="bf16x3", max_newton=3, max_iters=10, rank=20, wait_limit_ns=500_000_000)
    assert native.sync_status() == 0
    r = m.report
    assert r.device_bytes > 0
    assert r.device_bytes <= r.peak_bytes < torch.cuda.get_device_properties(0).total_memory
    m.free()
