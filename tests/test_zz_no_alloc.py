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


def _call_noalloc(native, A, B, S, Y, prec, ell, status):
    k = native.Kernel(native.KERNELS["matern32"], ell, 1.0)
    return native.lib.itergp_kmatvec_noalloc(
        ct.byref(k), native.PRECISIONS[prec], ct.c_void_p(A.data_ptr()), A.shape[0],
        ct.c_void_p(B.data_ptr()), B.shape[0], A.shape[1], ct.c_void_p(S.data_ptr()), S.shape[1],
        ct.c_void_p(Y.data_ptr()), ct.c_void_p(status.data_ptr()),
        ct.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16", "tf32"])
def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(native, prec):
    tol = 1e-4 if prec in ("fp32", "bf16x3", "tf32") else 1e-2
    g = np.random.default_rng(123)
    shapes = [(300, 517, 70, 21), (129, 260, 33, 80)]       # second call: other sizes
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    # every tensor the test touches is allocated before the first call
    cases = []
    for m, n, d, p in shapes:
        A = torch.as_tensor(g.standard_normal((m, d)), dtype=torch.float32, device=DEV)
        B = torch.as_tensor(g.standard_normal((n, d)), dtype=torch.float32, device=DEV)
        S = torch.as_tensor(g.standard_normal((n, p)), dtype=torch.float32, device=DEV)
        Y = torch.full((m, p), float("nan"), device=DEV)
        cases.append((A, B, S, Y, float(np.sqrt(d))))
    # a zero-size call performs the device set-up only
    assert _call_noalloc(native, cases[0][0][:0], cases[0][1], cases[0][2], cases[0][3], prec,
                         1.0, status) == 0
    first = []
    for A, B, S, Y, ell in cases:                            # two calls in a row
        rc = _call_noalloc(native, A, B, S, Y, prec, ell, status)
        assert rc == 0, native.status_string(rc)
    torch.cuda.synchronize()
    first = [c[3].clone() for c in cases]
    # the same two calls again: the device's free memory must not move (no allocation,
    # and every kernel they launch is loaded by now)
    free0 = torch.cuda.mem_get_info()[0]
    for A, B, S, Y, ell in cases:
        Y.fill_(float("nan"))
        rc = _call_noalloc(native, A, B, S, Y, prec, ell, status)
        assert rc == 0, native.status_string(rc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == 0
    for (A, B, S, Y, ell), Y1 in zip(cases, first):
        assert torch.isfinite(Y).all()
        assert torch.equal(Y, Y1)                            # the array kept no stale state
        Yr = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec)
        torch.cuda.synchronize()
        rel = (torch.linalg.norm(Y - Yr) / torch.linalg.norm(Yr)).item()
        assert rel <= tol, (prec, rel)


def test_noalloc_rejects_sizes_beyond_its_scratch(native):
    # rows padded to 30080 and d to 832: the BF16 hi and lo planes of A alone take
    # 30080 * 832 * 2 B * 2 = 95.5 MiB, above the 64 MiB array
    m = n = 30000
    A = torch.zeros((m, 784), device=DEV)
    S = torch.zeros((n, 8), device=DEV)
    Y = torch.full((m, 8), float("nan"), device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc = _call_noalloc(native, A, A, S, Y, "bf16x3", 28.0, status)
    assert rc == native.ESCRATCH
    assert "static buffer" in native.status_string(rc)
    torch.cuda.synchronize()
    assert torch.isnan(Y).all()         # nothing was launched
