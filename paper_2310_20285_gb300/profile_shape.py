"""Run one kernel-product shape repeatedly on the GPU (for profilers such as ncu).

    python -m paper_2310_20285_gb300.profile_shape --n 8192 --d 64 --p 16 \
        --precision bf16x3 --items --reps 5

--items runs the batched item schedule (one problem, every row tile an item), otherwise
the single-problem schedule of itergp_kmatvec.  Inputs are synthetic: X uniform in
[0, 1)^d, weights uniform in [-1, 1).  Prints the mean device time per launch.
"""
from __future__ import annotations

import argparse

import torch

from . import native


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--d", type=int, default=64)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--kind", default="rbf", choices=sorted(native.KERNELS))
    ap.add_argument("--precision", default="bf16x3", choices=sorted(native.PRECISIONS))
    ap.add_argument("--items", action="store_true")
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    if a.items:
        # itergp_autotune times every launch variant of the item schedule on this shape
        for _ in range(a.reps):
            vs, best = native.autotune(a.n, a.d, a.p, kind=a.kind, precision=a.precision, items=True)
        print({"variants_ms": vs, "best": best})
        return
    g = torch.Generator(device=dev).manual_seed(0)
    X = torch.rand((a.n, a.d), device=dev, generator=g)
    S = torch.rand((a.n, a.p), device=dev, generator=g) * 2 - 1
    Y = torch.empty((a.n, a.p), device=dev)
    native.kmatvec(X, X, S, kind=a.kind, precision=a.precision, out=Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        native.kmatvec(X, X, S, kind=a.kind, precision=a.precision, out=Y)
    e1.record()
    torch.cuda.synchronize()
    print({"ms_per_launch": e0.elapsed_time(e1) / a.reps})


if __name__ == "__main__":
    main()
