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


def force(native, tmp_path, prec, kind, d, p16, items, epi, stages, ares=-1):
    """Install one table entry through the text cache (ares: resident-A ring, one K slice
    only; -1 automatic)."""
    path = tmp_path / "tune.txt"
    d_pad = (d + 63) // 64 * 64
    path.write_text(f"{PREC_CODE[prec]} {kind} {d_pad} {p16} {items} {epi} {stages} {ares}\n")
    native.tune_clear()
    native.tune_load(path)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16_comp", "bf16", "tf32"])
@pytest.mark.parametrize("items,p", [(False, 16), (True, 16), (True, 128), (False, 80)])
def test_autotune_times_every_variant(native, prec, items, p):
    """Includes widths where the launchers tile P (128 split weights do not fit 2 stages)."""
    vs, best = native.autotune(4096, 32, p, precision=prec, items=items)
    assert len(vs) >= 2 and best in vs   # wide split P tiles leave room for 2 stages only
    assert {v[0] for v in vs} == {4, 8}
    assert all(v[2] > 0 for v in vs)
    native.tune_clear()


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("epi,stages,ares", [(8, 2, 0), (8, 4, 0), (4, 3, 0), (4, 3, 1), (8, 5, 1)])
def test_variants_compute_the_same_product(native, tmp_path, prec, epi, stages, ares):
    """D = 40 (one 64-wide K slice), so both the streamed and the resident-A rings apply
    (TF32 rows take two 32-wide slices and always stream; a resident-A entry falls back to
    the streamed ring); the reference is the streamed 4-warp ring."""
    X = torch.as_tensor(datagen.normal((3000, 40), 3), device=DEV)
    S = torch.as_tensor(datagen.normal((3000, 24), 4), device=DEV)
    force(native, tmp_path, prec, 1, 40, 32, 0, 4, 2, 0)
    ref = native.kmatvec(X, X, S, kind="matern32", lengthscale=3.0, precision=prec).clone()
    force(native, tmp_path, prec, 1, 40, 32, 0, epi, stages, ares)
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
