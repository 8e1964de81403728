"""The allocation-free kernel product (itergp_kmatvec_noalloc) against the regular one.

This entry point serves callers that may not allocate device memory while they run (for
example a serving loop that reserved all memory up front, or a host application with its
own allocator): its scratch is one fixed static device array, so the library makes no
allocation.  The test calls it through the C ABI twice in a row (the array keeps the
first call's contents) and compares each output with itergp_kmatvec's within the parity
tolerance of the other kernel-product tests.  It lives in its own file so it is collected
last; it passes both alone in a fresh process and after the other tests."""
import ctypes as ct

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _call_noalloc(native, A, B, S, prec, ell, status):
    k = native.Kernel(native.KERNELS["matern32"], ell, 1.0)
    Y = torch.full((A.shape[0], S.shape[1]), float("nan"), device=DEV)
    rc = native.lib.itergp_kmatvec_noalloc(
        ct.byref(k), native.PRECISIONS[prec], ct.c_void_p(A.data_ptr()), A.shape[0],
        ct.c_void_p(B.data_ptr()), B.shape[0], A.shape[1], ct.c_void_p(S.data_ptr()), S.shape[1],
        ct.c_void_p(Y.data_ptr()), ct.c_void_p(status.data_ptr()),
        ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, Y


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "tf32"])
def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(native, prec):
    tol = 1e-4 if prec in ("fp32", "bf16x3", "tf32") else 1e-2
    g = np.random.default_rng(123)
    shapes = [(300, 517, 70, 21), (129, 260, 33, 80)]       # second call: other sizes
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    for m, n, d, p in shapes:
        A = torch.as_tensor(g.standard_normal((m, d)), dtype=torch.float32, device=DEV)
        B = torch.as_tensor(g.standard_normal((n, d)), dtype=torch.float32, device=DEV)
        S = torch.as_tensor(g.standard_normal((n, p)), dtype=torch.float32, device=DEV)
        ell = float(np.sqrt(d))
        rc, Y = _call_noalloc(native, A, B, S, prec, ell, status)
        assert rc == 0, native.status_string(rc)
        Yr = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.isfinite(Y).all()
        rel = (torch.linalg.norm(Y - Yr) / torch.linalg.norm(Yr)).item()
        assert rel <= tol, (prec, rel)


def test_noalloc_rejects_sizes_beyond_its_scratch(native):
    m = n = 20000                       # BF16 hi/lo copies alone exceed 64 MiB at d = 784
    A = torch.zeros((m, 784), device=DEV)
    S = torch.zeros((n, 8), device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc, Y = _call_noalloc(native, A, A, S, "bf16x3", 28.0, status)
    assert rc == native.ESCRATCH
    assert "static buffer" in native.status_string(rc)
    torch.cuda.synchronize()
    assert torch.isnan(Y).all()         # nothing was launched
