"""Autotuned launch variants of the tensor-core product: the tuner times every variant
that fits, and every variant computes bitwise the same result (epilogue warps and stage
count only change which warp computes an element and how deep loads run ahead)."""
import numpy as np
import pytest
import torch

from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
PREC_CODE = {"bf16x3": 1, "bf16": 2, "bf16_comp": 3, "tf32": 4}


def force(native, tmp_path, prec, kind, d, p16, items, epi, stages, ares=-1, pair=-1):
    """Install one table entry through the text cache (ares: resident-A ring, one K slice
    only; pair: the CTA-pair form, single schedule only; -1 automatic)."""
    path = tmp_path / "tune.txt"
    d_pad = (d + 63) // 64 * 64
    path.write_text(f"{PREC_CODE[prec]} {kind} {d_pad} {p16} {items} {epi} {stages} {ares} {pair}\n")
    native.tune_clear()
    native.tune_load(path)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16_comp", "bf16", "tf32"])
@pytest.mark.parametrize("items,p", [(False, 16), (True, 16), (True, 128), (False, 80)])
def test_autotune_times_every_variant(native, prec, items, p):
    """Includes widths where the launchers tile P (128 split weights do not fit 2 stages)."""
    vs, best = native.autotune(4096, 32, p, precision=prec, items=items)
    assert len(vs) >= 2 and best in vs   # wide split P tiles leave room for 2 stages only
    assert {v[0] for v in vs} == {4, 8}
    assert all(v[3] > 0 for v in vs)
    # the pair form: single schedule; with wide chunks where P fits one tile of <= 80
    assert {v[2] for v in vs} == ({0} if items else {0, 1, 2} if p <= 80 else {0, 1})
    native.tune_clear()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("epi,stages,ares", [(8, 2, 0), (8, 4, 0), (4, 3, 0), (4, 3, 1), (8, 5, 1)])
def test_variants_compute_the_same_product(native, tmp_path, prec, epi, stages, ares):
    """D = 40 (one 64-wide K slice), so both the streamed and the resident-A rings apply
    (TF32 rows take two 32-wide slices and always stream; a resident-A entry falls back to
    the streamed ring); the reference is the streamed 4-warp ring."""
    X = torch.as_tensor(datagen.normal((3000, 40), 3), device=DEV)
    S = torch.as_tensor(datagen.normal((3000, 24), 4), device=DEV)
    force(native, tmp_path, prec, 1, 40, 32, 0, 4, 2, 0, 0)
    ref = native.kmatvec(X, X, S, kind="matern32", lengthscale=3.0, precision=prec).clone()
    force(native, tmp_path, prec, 1, 40, 32, 0, epi, stages, ares, 0)
    got = native.kmatvec(X, X, S, kind="matern32", lengthscale=3.0, precision=prec)
    native.tune_clear()
    assert torch.equal(got, ref)


@pytest.mark.parametrize("epi,stages,ares", [(8, 2, 0), (8, 3, 0), (4, 5, 1), (8, 3, 1)])
def test_variants_give_the_same_batched_fit(native, tmp_path, epi, stages, ares):
    probs = datagen.batch_problems(count=5, seed=17, n_lo=200, n_hi=1500, dims=(8, 16), c_lo=2,
                                   c_hi=7, ell_lo=0.8, ell_hi=3.0, n_test=16, ell_per_sqrt_d=True)
    dev = [(torch.as_tensor(p.X, device=DEV), torch.as_tensor(p.y, device=DEV), p.c, p.lengthscale, 1.0)
           for p in probs]
    sched = dict(max_newton=3, max_iters=6, rank=10, tol_abs=0.0, tol_rel=0.0)
    force(native, tmp_path, "bf16x3", 0, 16, 16, 1, 4, 2, 0)
    ref = native.fit_batch(dev, precision="bf16x3", **sched)
    force(native, tmp_path, "bf16x3", 0, 16, 16, 1, epi, stages, ares)
    got = native.fit_batch(dev, precision="bf16x3", **sched)
    native.tune_clear()
    for a, b in zip(got, ref):
        assert torch.equal(a.arrays()["f"], b.arrays()["f"])
        a.free()
        b.free()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16_comp", "bf16", "tf32"])
@pytest.mark.parametrize("m,n,d,p,epi,stages", [
    (3000, 3000, 40, 24, 4, 2),        # one K slice, three G buffers
    (2345, 1999, 300, 80, 8, 3),       # several slices, ragged rows, two G buffers
    (700, 4100, 784, 200, 8, 2),       # P split into tiles; tail rows shared by pairs
    (257, 300, 130, 16, 4, 4),         # one pair tile plus one row
])
def test_pair_form_computes_the_one_cta_product(native, tmp_path, prec, m, n, d, p, epi, stages):
    """The CTA-pair form (cta_group::2 MMAs of M = 256 issued for two SMs) issues the same
    MMAs per output element in the same order as the one-CTA form.  Only the split of the
    tail row tiles over CTAs (or pairs) differs, which regroups the FP32 partial sums of a
    row: the two agree to FP32 re-association (2^-18 of the row's largest output), far
    inside the 1e-4 product bar.  The ragged shapes exercise pair tiles past the last row
    and the tail fix-up."""
    A = torch.as_tensor(datagen.normal((m, d), 5), device=DEV)
    B = torch.as_tensor(datagen.normal((n, d), 6), device=DEV)
    S = torch.as_tensor(datagen.normal((n, p), 7), device=DEV)
    p16 = min((p + 15) // 16 * 16, 128)
    ell = float(np.sqrt(d))
    force(native, tmp_path, prec, 1, d, p16, 0, epi, stages, 0, 0)
    ref = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec).clone()
    force(native, tmp_path, prec, 1, d, p16, 0, epi, stages, 0, 1)
    got = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec)
    torch.cuda.synchronize()
    native.tune_clear()
    assert native.sync_status() == 0
    assert torch.isfinite(got).all()
    scale = ref.abs().amax(dim=1, keepdim=True).clamp_min(1e-30)
    err = float(((got - ref).abs() / scale).max())
    assert err <= 2.0 ** -18, err


@pytest.mark.parametrize("prec", ["bf16x3", "bf16_comp", "bf16", "tf32"])
@pytest.mark.parametrize("m,n,d,p,epi", [
    (3000, 3000, 40, 24, 4),           # one K slice
    (2345, 1999, 300, 80, 8),          # several slices, ragged rows, P = 80
    (700, 4100, 784, 80, 4),           # the kernel bench's D and P; a chunk past B's last row
    (257, 300, 130, 16, 8),            # one pair tile plus one row, two chunks
])
def test_wide_pair_form_computes_the_one_cta_product(native, tmp_path, prec, m, n, d, p, epi):
    """The wide pair form (chunks of 192 rows of B, MMA N = 192, the flushed running sum in
    registers) forms each kernel value and weighted-sum term as the one-CTA form does;
    its chunks and flush groups (3 x 192 rather than 4 x 128 rows) regroup the FP32 sums
    of a row, so the two agree to FP32 re-association (2^-16 of the row's largest output,
    far inside the 1e-4 product bar).  Chunks past the last row of B read zero rows,
    norms and weights."""
    A = torch.as_tensor(datagen.normal((m, d), 5), device=DEV)
    B = torch.as_tensor(datagen.normal((n, d), 6), device=DEV)
    S = torch.as_tensor(datagen.normal((n, p), 7), device=DEV)
    p16 = (p + 15) // 16 * 16
    ell = float(np.sqrt(d))
    force(native, tmp_path, prec, 1, d, p16, 0, epi, 2, 0, 0)
    ref = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec).clone()
    force(native, tmp_path, prec, 1, d, p16, 0, epi, 3, 0, 2)
    got = native.kmatvec(A, B, S, kind="matern32", lengthscale=ell, precision=prec)
    torch.cuda.synchronize()
    native.tune_clear()
    assert native.sync_status() == 0
    assert torch.isfinite(got).all()
    scale = ref.abs().amax(dim=1, keepdim=True).clamp_min(1e-30)
    err = float(((got - ref).abs() / scale).max())
    assert err <= 2.0 ** -16, err


def test_wide_pair_form_keeps_the_exact_diagonal(native, tmp_path):
    """K(X, X) S with the wide chunks: 192-row chunks straddle the 256-row pair tiles, so a
    row's own column falls at any offset of a chunk; the kernel value there is s (to the
    exp2 and FP16-split rounding, 2^-20), where |a|^2 + |a|^2 - 2 a.a in split FP16 would
    leave about 3e-3 in r^2 and e^-0.6 in k.  The kernel is so narrow (|x| ~ 80, l = 0.05)
    that every other value underflows to 0: K = s I."""
    X = torch.as_tensor(datagen.normal((1000, 64), 8) * 10.0, device=DEV)
    S = torch.as_tensor(datagen.normal((1000, 16), 9), device=DEV)
    force(native, tmp_path, "bf16x3", 0, 64, 16, 0, 4, 3, 0, 2)
    got = native.kmatvec(X, X, S, kind="rbf", lengthscale=0.05, outputscale=2.5, precision="bf16x3")
    torch.cuda.synchronize()
    native.tune_clear()
    assert native.sync_status() == 0
    want = 2.5 * S
    err = float(((got - want).abs() / want.abs().amax(dim=1, keepdim=True)).max())
    assert err <= 2.0 ** -20, err
