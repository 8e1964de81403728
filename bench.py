#!/usr/bin/env python
"""Benchmark of the IterNCGP hot path on GB300; prints one JSON line.

Step = one kernel product K(X, X) S on the kernel-bench workload (N = 60000 points of
784-D sparse clusters, Matern-3/2 l = 28, S of N x 80 standard normals), computed through
the C ABI (itergp_kmatvec) in the FP32-accurate tensor-core precision (bf16x3).  The
metric is kernel pairs per second (N^2 / step time).  The same JSON line carries the
end-to-end number (host buffers, copies inside the timed region), the roofline of the
fused product kernel, the other precisions, Newton-step times of the full fit on the
same data (plain FP32 path vs tensor-core paths), clocks sampled during the timed region
and the FP64 oracle's throughput on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT, D, P = 60000, 784, 80
ELL, OUT = 28.0, 1.0
METRIC = "K·S kernel-pairs/s"


# ---- the N > 1 path: independent replicas (weak scaling), no data-path collective
def replica_seed(rank: int) -> int:
    """Each rank draws its own independent problem of the same shape."""
    return 2 + 1000 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (an all-reduce MAX over the process group; the value
    itself for a single process)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: every rank processes its own units within the slowest rank's
    time."""
    return world * units_per_rank / t_max


def guarded(fn, *args, **kwargs):
    """An extra section's result, or its error as {"error": ...}: the headline JSON line
    must not depend on the sections printed beside it."""
    try:
        return fn(*args, **kwargs)
    except Exception as e:   # noqa: BLE001 -- reported in the line, never swallowed silently
        return {"error": f"{type(e).__name__}: {str(e)[:300]}"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-extras", action="store_true", help="skip other precisions and fit timings")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-count", type=int, default=256, help="problems of the batched-fit extra")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the serving extra")
    ap.add_argument("--no-tune", action="store_true", help="skip autotuning the product's launch variants")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return summarize_clock_samples(lines)


def summarize_clock_samples(lines):
    """Median SM clock, maximum clock and the throttle reasons seen in `nvidia-smi` CSV rows
    of the FIELDS above (no header, no units)."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(X, S, seconds: float):
    """The FP64 oracle's k(X, X) S on a bounded sample of output rows (host cores)."""
    import numpy as np

    import oracle.itergp_oracle as O
    kern = O.Kernel(O.MATERN32, ELL, OUT)
    X64 = X.astype(np.float64)
    S64 = S.astype(np.float64)
    rows, t0 = 0, time.perf_counter()
    chunk = 64
    while time.perf_counter() - t0 < seconds and rows < X.shape[0]:
        O.kmatvec(X64[rows:rows + chunk], X64, S64, kern)
        rows += chunk
    dt = time.perf_counter() - t0
    return {"value": rows * X.shape[0] / dt, "unit": "kernel-pairs/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{rows} of {X.shape[0]} output rows of k(X,X)S (FP64 NumPy, D={X.shape[1]}, P={S.shape[1]})",
            "seconds": round(dt, 2)}


def newton_step_ms_small(native, datagen, torch, dev, reps=5):
    """The small multi-class workload (N = 500 blobs, D = 2, C = 3, RBF l = 1, 10 Newton
    steps x <= 50 CG iterations, R = 50, tolerances 1e-5) on the GPU: ms per Newton step of
    whole fits (median of `reps`, after one warm-up), FP32 against BF16X3, with the fit
    captured into one CUDA graph and with direct launches."""
    import numpy as np
    X, y, _, _ = datagen.workload_small()
    tX = torch.as_tensor(X.astype(np.float32), device=dev)
    ty = torch.as_tensor(y, device=dev)
    out = {"workload": "N=500, D=2, C=3 blobs, RBF l=1, 10 Newton x <=50 CG, R=50, tol 1e-5"}
    for prec in ("fp32", "bf16x3"):
        row = {}
        for graph in (True, False):
            ts, steps = [], 10
            for r in range(reps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m = native.fit(tX, ty, 3, kind="rbf", lengthscale=1.0, precision=prec, max_newton=10,
                               max_iters=50, rank=50, graph=graph)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                steps = int(m.report.newton_steps)
                m.free()
                if r > 0:
                    ts.append(dt)
            row["graph" if graph else "direct"] = {"newton_step_ms": round(float(np.median(ts)) * 1e3 / steps, 4),
                                                    "fit_ms": round(float(np.median(ts)) * 1e3, 3)}
        out[prec] = row
    return out


def cpu_baseline_oracle_runs(native, datagen, torch, dev, X, S, seconds):
    """The FP64 oracle beyond the headline product, on the host cores, and the error of
    every GPU result against it:
      - the small workload's full fit (10 x 50, R = 50) timed;
      - the precision report of the 5000-point inputs (the small workload's generator at
        N = 5000 and the first 5000 rows of the kernel-bench data): K.S (24 columns), every
        Newton iterate f_i and the predictive mean of a 10 x 50, R = 50 fit, per precision;
      - the kernel-bench fit (N = 60000, 5 Newton x 5 iterations, R = 200) estimated from
        the oracle's own pieces timed on a row block: its dense kernel matrix and its K
        products (the solver's O(N C B) work is small next to them);
      - the oracle's FP32 matrix-free product on a row sample."""
    import numpy as np

    import oracle.itergp_oracle as O
    res = {}
    X1, y1, _, _ = datagen.workload_small()
    t0 = time.perf_counter()
    O.iterncgp_fit(X1.astype(np.float32).astype(np.float64), O.Softmax(y1, 3), 3, O.Kernel(O.RBF, 1.0, 1.0),
                   max_newton=10, max_iters=50, R=50)
    res["small_fit_s"] = round(time.perf_counter() - t0, 3)

    def rel(a, b):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    precs = ["fp32", "bf16x3", "bf16_comp", "bf16", "tf32"]
    acc = {"workload": "5000-point inputs: blobs (the small workload's generator, D=2, RBF l=1) and "
                       "the first 5000 rows of the kernel-bench data (D=784, Matern l=28); errors are "
                       "normwise relative against the FP64 oracle"}
    for data in ("blobs5000", "kernel_bench5000"):
        if data == "blobs5000":
            Xa, ya, Xsa, _ = datagen.blobs_train_test(5000, 200, d=2, c=3, seed=0)
            kern, kind = O.Kernel(O.RBF, 1.0, 1.0), "rbf"
        else:
            Xa, ya, Xsa, _, _ = datagen.workload_kernel_bench(n=5000, n_test=10)
            kern, kind = O.Kernel(O.MATERN32, 28.0, 1.0), "matern32"
        Xa = np.asarray(Xa, dtype=np.float32)
        Sa = datagen.normal((5000, 24), 77)
        t0 = time.perf_counter()
        ref = O.kmatvec(Xa.astype(np.float64), Xa.astype(np.float64), Sa.astype(np.float64), kern)
        res[f"kmatvec_{data}_s"] = round(time.perf_counter() - t0, 3)
        tX, tS = torch.as_tensor(Xa, device=dev), torch.as_tensor(Sa, device=dev)
        acc[f"K.S {data}"] = {p: rel(native.kmatvec(tX, tX, tS, kind=kind, lengthscale=kern.lengthscale,
                                                     precision=p).cpu(), ref) for p in precs}
        if data == "blobs5000":
            t0 = time.perf_counter()
            fref = O.iterncgp_fit(Xa.astype(np.float64), O.Softmax(ya, 3), 3, kern, max_newton=10,
                                  max_iters=50, R=50)
            res["blobs5000_fit_s"] = round(time.perf_counter() - t0, 3)
            em, _, _ = O.predict(Xsa.astype(np.float32).astype(np.float64), Xa.astype(np.float64), fref.v,
                                 fref.Q, kern, 3)
            ty = torch.as_tensor(ya, device=dev)
            tXs = torch.as_tensor(Xsa.astype(np.float32), device=dev)
            fit = {}
            for p in precs:
                fi, mean_err = [], None
                for i in range(1, 11):
                    m = native.fit(tX, ty, 3, kind="rbf", lengthscale=1.0, precision=p, max_newton=i,
                                   max_iters=50, rank=50)
                    fi.append(rel(m.arrays()["f"].cpu(), fref.fs[i]))
                    if i == 10:
                        mean, _, _ = m.predict(tXs)
                        mean_err = rel(mean.cpu(), em)
                    m.free()
                fit[p] = {"f_i": [float(f"{e:.3g}") for e in fi], "mean": mean_err}
            acc["fit blobs5000 (10 x 50, R=50)"] = fit
    res["accuracy"] = acc
    # kernel-bench fit, estimated from the oracle's own pieces on a row block
    n = X.shape[0]
    blk = 1000
    kern2 = O.Kernel(O.MATERN32, ELL, OUT)
    X64 = X.astype(np.float64)
    t0 = time.perf_counter()
    Kb = O.kernel_matrix(X64[:blk], X64, kern2)
    t_k = time.perf_counter() - t0
    W = np.asarray(S[:, :10], dtype=np.float64)
    t0 = time.perf_counter()
    for _ in range(3):
        Kb @ W
    t_p = (time.perf_counter() - t0) / 3
    products = 5 * 5 + 5   # one K product per solver iteration plus f = K v per Newton step
    est = (t_k + products * t_p) * n / blk
    res["kernel_bench_fit_s_estimated"] = {"value": round(est, 1), "kernel_matrix_s": round(t_k * n / blk, 1),
                                           "products": products, "product_s": round(t_p * n / blk, 3),
                                           "note": f"oracle pieces timed on {blk} of {n} rows and scaled by rows; "
                                                   "the dense K it builds holds 28.8 GB in FP64"}
    # the oracle's FP32 matrix-free product
    rows, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and rows < n:
        O.kmatvec_fp32(X[rows:rows + 64], X, S, kern2)
        rows += 64
    dt = time.perf_counter() - t0
    res["kmatvec_fp32"] = {"value": rows * n / dt, "unit": "kernel-pairs/s", "cores": os.cpu_count(),
                           "sample": f"{rows} of {n} output rows (FP32 NumPy, D={X.shape[1]}, P={S.shape[1]})",
                           "seconds": round(dt, 2)}
    return res


_ONE_CORE_CHILD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle.itergp_oracle as O
from paper_2310_20285_gb300 import datagen
n, seconds, ell, out = int(sys.argv[2]), float(sys.argv[3]), float(sys.argv[4]), float(sys.argv[5])
X, _, _, _, S = datagen.workload_kernel_bench(n=n)
X64, S64 = X.astype(np.float64), S.astype(np.float64)
kern = O.Kernel(O.MATERN32, ell, out)
rows, t0 = 0, time.perf_counter()
while time.perf_counter() - t0 < seconds and rows < n:
    O.kmatvec(X64[rows:rows + 64], X64, S64, kern)
    rows += 64
dt = time.perf_counter() - t0
print(json.dumps({"rows": rows, "seconds": dt}))
"""


def cpu_baseline_one_core(n: int, seconds: float):
    """The same oracle product on one host core: a child process with every BLAS/OpenMP
    pool limited to one thread (the pools size themselves when NumPy loads).  Never raises;
    a failure is reported in the result."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _ONE_CORE_CHILD, ROOT, str(n), str(seconds), str(ELL), str(OUT)],
                           env=env, capture_output=True, text=True, timeout=seconds + 180)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": d["rows"] * n / d["seconds"], "unit": "kernel-pairs/s", "cores": 1,
                "sample": f"{d['rows']} of {n} output rows (FP64 NumPy, BLAS and OpenMP pools of one thread)",
                "seconds": round(d["seconds"], 2)}
    except Exception as e:   # the bench line must not depend on this side measurement
        return {"error": f"{type(e).__name__}: {str(e)[:200]}"}


def reference_arm(args):
    """Oracle on the host cores as the reference implementation (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2310_20285_gb300 import datagen
    X, _, _, _, S = datagen.workload_kernel_bench(n=args.n)
    import numpy as np

    import oracle.itergp_oracle as O
    kern = O.Kernel(O.MATERN32, ELL, OUT)
    X64, S64 = X.astype(np.float64), S.astype(np.float64)
    rows_per_step = 32
    for w in range(args.warmup):
        O.kmatvec(X64[:8], X64, S64, kern)
    times = []
    for k in range(args.steps):
        r0 = (k * rows_per_step) % X.shape[0]
        t0 = time.perf_counter()
        O.kmatvec(X64[r0:r0 + rows_per_step], X64, S64, kern)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = rows_per_step * X.shape[0] / t
    out = {"metric": METRIC, "value": value, "unit": "kernel-pairs/s", "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"kernel product K(X,X)S, N={args.n}, D={D}, P={P}, Matern-3/2 l=28 "
                                  f"(bounded sample: {rows_per_step} output rows per step)"},
           "cpu_baseline": {"value": value, "unit": "kernel-pairs/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"{rows_per_step} output rows of k(X,X)S per step"},
           "e2e": {"value": value, "unit": "kernel-pairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


BATCH_SCHED = dict(max_newton=5, max_iters=5, rank=50, tol_abs=1e-5, tol_rel=1e-5)


def bench_batched(native, datagen, torch, dev, count):
    """Batched fits: `count` independent blob problems (N log-uniform in [200, 20000],
    D in {8, 16, 32, 64}, C in {2..10}, RBF lengthscale log-uniform in [0.3, 3]), one
    schedule of 5 Newton steps x <= 5 iterations, R = 50, tolerance 1e-5.  Each batched
    fit is one itergp_fit_batch call (graph captured and launched inside); the plain
    path fits the same problems one by one in FP32 without a graph."""
    probs = datagen.batch_problems(count=count)
    dp = [(torch.as_tensor(p.X, device=dev), torch.as_tensor(p.y, device=dev), p.c,
           p.lengthscale, 1.0) for p in probs]
    n = [p.X.shape[0] for p in probs]
    res = {"workload": f"{count} blob problems, N log-U[200,20000] (sum {sum(n)}), D in {{8,16,32,64}}, "
                       "C in {2..10}, RBF l log-U[0.3,3]; 5 Newton x <=5 iters, R=50, tol 1e-5",
           "sum_n2": float(sum(x * x for x in n))}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        models = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, models

    for prec in ("fp32", "bf16x3", "bf16_comp"):
        try:
            for m in native.fit_batch(dp, precision=prec, graph=True, errors="return", **BATCH_SCHED):
                if isinstance(m, native.Model):   # warm-up
                    m.free()
            l0 = native.launch_count()
            dt, models = timed(lambda: native.fit_batch(dp, precision=prec, graph=True, errors="return",
                                                        **BATCH_SCHED))
            launches = native.launch_count() - l0
        except native.ItergpError as e:
            res[prec] = {"error": str(e)}
            continue
        ok = [(m, x) for m, x in zip(models, n) if isinstance(m, native.Model)]
        iters = [m.report.total_iters for m, _ in ok]
        pairs = float(sum(m.report.total_iters * x * x for m, x in ok))
        res[prec] = {"fit_s": dt, "fits_per_s": count / dt, "total_iters": int(sum(iters)),
                     "kernel_pairs_per_s": pairs / dt, "launches": int(launches),
                     "failed": [str(m) for m in models if not isinstance(m, native.Model)]}
        for m, _ in ok:
            m.free()
    l0 = native.launch_count()
    t0 = time.perf_counter()
    it_plain = 0
    for X_, y_, c_, ell_, s_ in dp:
        m = native.fit(X_, y_, c_, kind="rbf", lengthscale=ell_, outputscale=s_, precision="fp32",
                       graph=False, **BATCH_SCHED)
        it_plain += m.report.total_iters
        m.free()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res["fp32_one_by_one"] = {"fit_s": dt, "fits_per_s": count / dt, "total_iters": int(it_plain),
                              "launches": int(native.launch_count() - l0)}
    return res


def small_d_roofline(native, torch, dev, n=131072, d=32, p=16):
    """The product at small D (the batched and served shapes) is bound by the exp per
    kernel value, not by the tensor cores: 2 (D + P) tensor flops against one MUFU exp2
    per pair (RBF).  Measured against this GPU's MUFU exp2 and FFMA rates, probed here."""
    ex2 = native.probe_throughput("ex2")
    ffma = native.probe_throughput("ffma")
    g = torch.Generator(device=dev).manual_seed(0)
    X = torch.rand((n, d), device=dev, generator=g) * 4.0
    S = torch.rand((n, p), device=dev, generator=g) * 2 - 1
    Y = torch.empty((n, p), device=dev)
    res = {"probe_ex2_per_s": ex2, "probe_ffma_flops_per_s": ffma,
           # the other units the product's forms use, probed the same way
           "probe_rsqrt_per_s": native.probe_throughput("rsqrt"),
           "probe_dfma_flops_per_s": native.probe_throughput("dfma"),
           "probe_mma_tf32_flops_per_s": native.probe_throughput("mma_ss_n128_tf32"),
           "probe_mma_bf16_flops_per_s": native.probe_throughput("mma_ss_n128"),
           "shape": f"single product N={n}, D={d}, P={p}, RBF, inputs U[0,4)^D"}
    for prec in ("bf16x3", "bf16_comp", "fp32"):
        native.kmatvec(X, X, S, kind="rbf", lengthscale=1.0, precision=prec, out=Y)
        torch.cuda.synchronize()
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            native.kmatvec(X, X, S, kind="rbf", lengthscale=1.0, precision=prec, out=Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        pairs = n * n / (ms * 1e-3)
        res[prec] = {"ms": ms, "kernel_pairs_per_s": pairs,
                     "roofline": {"bound": "sfu", "achieved": pairs, "peak": ex2, "unit": "exp2/s",
                                  "frac": pairs / ex2, "peak_kind": "measured here (ex2.approx probe)"}}
    return res


def calibration_metrics(probs, y, n_bins=15):
    """Accuracy, NLL (negative mean log-probability of the true class) and expected
    calibration error of the top-class confidence over n_bins equal-width bins."""
    import numpy as np
    probs = np.asarray(probs, dtype=np.float64)
    pred = probs.argmax(1)
    conf = probs.max(1)
    correct = (pred == y).astype(np.float64)
    nll = float(-np.mean(np.log(np.maximum(probs[np.arange(len(y)), y], 1e-300))))
    edges = np.linspace(0.0, 1.0, n_bins + 1)
    ece = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (conf > lo) & (conf <= hi)
        if m.any():
            ece += m.mean() * abs(correct[m].mean() - conf[m].mean())
    return float(correct.mean()), nll, float(ece)


def bench_gmm(native, datagen, torch, dev):
    """The paper's large-scale synthetic problem (App. C.3): 10 classes of 3-D Gaussians,
    10^4 training points per class (N = 10^5), 10^3 test points per class, Matern-3/2
    l = 0.05, s = 0.05, CG actions with recycling, j <= 5, R = infinity and R = 10.  Each
    row is a fit stopped after k Newton steps (timed), then test accuracy, NLL and ECE
    (15 bins) of the probit predictive, computed outside the timed region."""
    import numpy as np
    X, y = datagen.gmm3d(10000, seed_model=1, seed_draw=2)
    Xs, ys = datagen.gmm3d(1000, seed_model=1, seed_draw=3)
    tX = torch.as_tensor(X.astype(np.float32), device=dev)
    ty = torch.as_tensor(y, device=dev)
    tXs = torch.as_tensor(Xs.astype(np.float32), device=dev)
    out = {"workload": "GMM, C=10, D=3, N=1e5 train / 1e4 test, Matern-3/2 l=0.05 s=0.05, "
                       "CG actions, recycling, j<=5; fits stopped after k Newton steps",
           "runs": []}
    for prec, rank in (("bf16x3", None), ("bf16x3", 10), ("fp32", 10)):
        rows = []
        for k in (1, 2, 3, 5, 8):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                m = native.fit(tX, ty, 10, kind="matern32", lengthscale=0.05, outputscale=0.05,
                               precision=prec, max_newton=k, max_iters=5, rank=rank)
            except native.ItergpError as e:
                rows.append({"newton_steps": k, "error": str(e)})
                break
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            _, _, probs = m.predict(tXs)
            acc, nll, ece = calibration_metrics(probs.cpu().numpy(), ys)
            rows.append({"newton_steps": k, "fit_s": round(dt, 4), "test_acc": round(acc, 4),
                         "test_nll": round(nll, 4), "test_ece": round(ece, 4),
                         "iters": int(m.report.total_iters)})
            m.free()
        out["runs"].append({"precision": prec, "R": "inf" if rank is None else rank, "by_steps": rows})
    return out


def bench_class_kernels(native, datagen, torch, dev):
    """One kernel per output GP on the paper's Gaussian-mixture data (C = 10, D = 3,
    N = 10^5): the product K S for an N x C block with per-class Matern-3/2 lengthscales
    l_c = 0.05 (1 + 0.1 c) (grouped: C products of one column each) against the shared
    kernel (one product of C columns), and a fit on 20000 training points (5 Newton x 5
    iterations, R = 10) with per-class against shared hyperparameters, test accuracy on
    the 10^4 test points outside the timed region."""
    import numpy as np
    X, y = datagen.gmm3d(10000, seed_model=1, seed_draw=2)
    Xs, ys = datagen.gmm3d(1000, seed_model=1, seed_draw=3)
    tX = torch.as_tensor(X.astype(np.float32), device=dev)
    tXs = torch.as_tensor(Xs.astype(np.float32), device=dev)
    n = tX.shape[0]
    ks = [("matern32", 0.05 * (1 + 0.1 * c), 0.05) for c in range(10)]
    g = torch.Generator(device=dev).manual_seed(0)
    S = torch.randn((n, 10), device=dev, generator=g)
    Y = torch.empty_like(S)
    out = {"workload": "GMM C=10 D=3; product N=1e5, S N x 10; fit N=2e4 (first 2000 per class), "
                       "5 Newton x 5 iters, R=10, bf16x3; per-class l_c = 0.05 (1 + 0.1 c), s = 0.05"}

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_cls = timed(lambda: native.kmatvec_classes(tX, tX, S, ks, precision="bf16x3", out=Y))
    t_sh = timed(lambda: native.kmatvec(tX, tX, S, kind="matern32", lengthscale=0.05, outputscale=0.05,
                                        precision="bf16x3", out=Y))
    out["product"] = {"per_class_ms": t_cls, "shared_ms": t_sh,
                      "per_class_kernel_values_per_s": 10 * n * n / (t_cls * 1e-3),
                      "shared_kernel_values_per_s": n * n / (t_sh * 1e-3)}
    sub = np.concatenate([np.where(y == c)[0][:2000] for c in range(10)])
    tXf = torch.as_tensor(X[sub].astype(np.float32), device=dev)
    tyf = torch.as_tensor(y[sub], device=dev)
    fits = {}
    for label, kw in (("per_class", dict(class_kernels=ks)),
                      ("shared", dict(kind="matern32", lengthscale=0.05, outputscale=0.05))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = native.fit(tXf, tyf, 10, precision="bf16x3", max_newton=5, max_iters=5, rank=10, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        _, _, probs = m.predict(tXs)
        acc, nll, ece = calibration_metrics(probs.cpu().numpy(), ys)
        fits[label] = {"fit_s": round(dt, 4), "test_acc": round(acc, 4), "test_nll": round(nll, 4),
                       "test_ece": round(ece, 4), "iters": int(m.report.total_iters)}
        m.free()
    out["fit"] = fits
    return out


def bench_likelihoods(native, datagen, torch, dev, n=20000, n_test=10000):
    """The one-latent likelihoods and the conjugate case through the same Alg. 1-3 path,
    BF16X3, on N = 2e4 points X ~ U[-3, 3]^2 with g(x) = sin(x_1) + x_2 / 2:
    Bernoulli with the logistic link (App. C; labels drawn with P(y = 1) = sigma(2 g)),
    RBF l = 0.5, s = 0.2, 8 Newton steps x 5 CG iterations, R = 10; Poisson with the log
    link (App. A; y ~ Poisson(e^g)), RBF l = 0.3, s = 0.05, started at the constant
    f_0 = log(mean y), 8 x 5, R = 10; the Gaussian likelihood (Thm. A.2; noise variance
    0.01), RBF l = 1, s = 1, one Newton step of 50 iterations without truncation (the FP64
    oracle's test RMSE is 1.9 after 20 iterations and 0.063 after 50).
    The undamped Newton iteration of Alg. 1 diverges on these data at larger kernel
    scales (the FP64 oracle too, e.g. l = 1, s = 1, or any s >= 0.2 for Poisson at
    N >= 1.6e4), so the scales are ones the oracle converges on at this N.  Each row:
    fit wall time, predictive time on 1e4 test points (CUDA events, mean of 5), and the
    test RMSE of the predictive mean against the latent the labels were drawn from."""
    import numpy as np
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"one latent, N={n:g} train / {n_test:g} test, D=2, X ~ U[-3,3]^2, "
                       "g = sin(x1) + x2/2, RBF, bf16x3"}
    setups = {"bernoulli": (0.5, 0.2, dict(max_newton=8, max_iters=5, rank=10)),
              "poisson": (0.3, 0.05, dict(max_newton=8, max_iters=5, rank=10)),
              "gaussian": (1.0, 1.0, dict(max_newton=1, max_iters=50, rank=-1, noise=0.01))}
    for kind, (ell, sc, kw) in setups.items():
        X, y, Xs = datagen.one_latent(kind, n, seed=11, n_test=n_test)
        g_test = np.sin(Xs[:, 0].astype(np.float64)) + 0.5 * Xs[:, 1]
        latent = 2.0 * g_test if kind == "bernoulli" else g_test
        tX = torch.as_tensor(X, device=dev)
        tXs = torch.as_tensor(Xs, device=dev)
        ty = torch.as_tensor(y.reshape(-1, 1) if kind == "gaussian" else y, device=dev)
        if kind == "poisson":
            kw = dict(kw, f0=torch.full((n, 1), float(np.log(y.mean())), device=dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = native.fit(tX, ty, 1, kind="rbf", lengthscale=ell, outputscale=sc, likelihood=kind,
                       precision="bf16x3", **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        m.predict(tXs)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            mean, _, _ = m.predict(tXs)
        e1.record()
        torch.cuda.synchronize()
        mu = mean.double().cpu().numpy().reshape(-1)
        r = m.report
        out[kind] = {"lengthscale": ell, "outputscale": sc, "fit_s": round(dt, 4),
                     "newton_steps": int(r.newton_steps), "iters": int(r.total_iters),
                     "objective": [round(r.objective[i], 1) for i in range(r.newton_steps)],
                     "predict_ms": round(e0.elapsed_time(e1) / 5, 3),
                     "test_rmse_mean_vs_latent": round(float(np.sqrt(np.mean((mu - latent) ** 2))), 4)}
        m.free()
    return out


def mc_nll(mu, var, y, samples, rng):
    """Monte-Carlo negative log predictive density of Poisson counts y under latent
    N(mu, var) per point (App. C): -log mean_k Poisson(y | e^{f_k}), averaged over the
    points."""
    import numpy as np
    from math import lgamma
    z = rng.standard_normal((samples, 1))
    f = mu[None, :] + np.sqrt(np.maximum(var, 0.0))[None, :] * z       # samples x n
    lp = y[None, :] * f - np.exp(f) - np.array([lgamma(v + 1.0) for v in y])[None, :]
    mx = lp.max(axis=0)
    return float(np.mean(-(mx + np.log(np.mean(np.exp(lp - mx), axis=0)))))


def bench_poisson_study(native, datagen, torch, dev, runs=10, samples=10000):
    """The Poisson-regression budget study (App. C): 100 points in [0, 1], a log-rate drawn
    from an RBF GP (l = 0.1, s = 5), counts y ~ Poisson(e^f); the prior uses the same
    kernel.  A budget of 100 solver iterations is spread over 5, 10, 20 or 100 Newton steps
    (j <= 20, 10, 5, 1), CG actions with recycling and no compression, outer tolerance
    0.001; `runs` training sets re-drawn at the same rates, and a test set drawn the same
    way.  Fits run through itergp_fit (Poisson likelihood, FP32); the NLL is a Monte-Carlo
    estimate over `samples` draws per point, outside the timed region, summarised as the
    figure does (median, min and max over the runs).  Two starts: f_0 = m = 0 as Alg. 1
    prints it, and the constant f_0 = log(mean y).  The undamped Newton iteration
    overshoots on some training sets (from 0 with j <= 10 or 20; at j <= 5 on some sets
    from either start), and the FP64 oracle does the same on them."""
    import numpy as np
    X, f_true, Y, Yt = datagen.poisson_study(seed=11, runs=runs)
    tX = torch.as_tensor(X, device=dev)
    rng = np.random.default_rng(12)
    out = {"workload": f"Poisson regression, N=100 in [0,1], RBF l=0.1 s=5, {runs} runs, budget 100 "
                       f"solver iterations, outer tol 1e-3, R unbounded, fp32; MC-NLL with {samples} "
                       "draws per point (the paper uses 1e5)"}
    def stats(v):   # the figure's statistics: median and min / max over the runs
        if not v:
            return None
        return {"median": round(float(np.median(v)), 4), "min": round(float(np.min(v)), 4),
                "max": round(float(np.max(v)), 4)}

    for start in ("zero", "log_mean"):
        rows = {}
        for steps in (5, 10, 20, 100):
            j = 100 // steps
            tr, te, ms, used, errs = [], [], [], [], []
            for r in range(runs):
                ty = torch.as_tensor(Y[r], device=dev)
                kw = {}
                if start == "log_mean":
                    kw["f0"] = torch.full((100, 1), float(np.log(max(Y[r].mean(), 1e-3))), device=dev)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    m = native.fit(tX, ty, 1, kind="rbf", lengthscale=0.1, outputscale=5.0, likelihood="poisson",
                                   precision="fp32", max_newton=steps, max_iters=j, rank=-1, tol_newton=1e-3, **kw)
                except native.ItergpError as e:
                    errs.append(str(e)[:60])
                    continue
                torch.cuda.synchronize()
                ms.append((time.perf_counter() - t0) * 1e3)
                used.append(int(m.report.newton_steps))
                mean, var, _ = m.predict(tX)
                mu = mean.double().cpu().numpy().reshape(-1)
                vv = var.double().cpu().numpy().reshape(-1)
                m.free()
                if not np.all(np.isfinite(mu)):
                    errs.append("non-finite predictive mean")
                    continue
                tr.append(mc_nll(mu, vv, Y[r].astype(np.float64), samples, rng))
                te.append(mc_nll(mu, vv, Yt[r].astype(np.float64), samples, rng))
            rows[f"{steps}x{j}"] = {
                "runs_ok": len(tr), "failed": errs[:3] + ([f"... {len(errs) - 3} more"] if len(errs) > 3 else []),
                "train_nll": stats(tr), "test_nll": stats(te),
                "fit_ms": round(float(np.mean(ms)), 3) if ms else None,
                "newton_steps_used": [int(min(used)), int(max(used))] if used else None}
        out[f"start_{start}"] = rows
    return out


def bench_serving(native, datagen, precision, seconds, seed=5, drain_s=10.0):
    """Serving: Poisson arrivals over `seconds` of fit requests at 50/s (N log-uniform in
    [1e3, 5e4], D = 32, C = 5 blobs, RBF l log-uniform in [0.3, 3]; 5 Newton x <= 5
    iterations, R = 50) and predict requests at 2000/s (M uniform in [1, 4096], D = 32)
    against models already resident, admitted under an 80 GB model budget.  The fit
    inputs come from a pool of 64 generated problems and the queries from a pool of 16
    blocks (every request is still its own copy, fit and model).  Latency = completion
    (results in the caller's host buffers) minus submission."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pool = datagen.batch_problems(count=64, seed=seed, n_lo=1000, n_hi=50000, dims=(32,), c_lo=5,
                                  c_hi=5, ell_lo=0.3, ell_hi=3.0, n_test=8)
    qpool = [datagen.normal((4096, 32), seed + 100 + k) * 3.0 for k in range(16)]
    fit_t = np.cumsum(rng.exponential(1 / 50.0, size=int(60 * seconds) + 10))
    pred_t = np.cumsum(rng.exponential(1 / 2000.0, size=int(2100 * seconds) + 10))
    fit_t = fit_t[fit_t < seconds]
    pred_t = pred_t[pred_t < seconds]
    arrivals = sorted([(t, 0) for t in fit_t] + [(t, 1) for t in pred_t])
    fit_pick = rng.integers(0, len(pool), size=len(fit_t))
    pred_m = rng.integers(1, 4097, size=len(pred_t))
    pred_q = rng.integers(0, len(qpool), size=len(pred_t))
    pred_u = rng.random(size=len(pred_t))
    srv = native.Server(model_bytes=80 << 30, work_bytes=24 << 30, precision=precision, d_max=32,
                        c_max=5, max_fit_batch=64, max_predict_batch=512, max_predict_rows=1 << 18,
                        max_newton=5, max_iters=5, rank=50, graph=True)
    resident, lat = [], {0: [], 1: []}
    queue, service = {0: [], 1: []}, {0: [], 1: []}   # submission -> start, start -> done
    done_fit, skipped, kinds = 0, 0, {}
    submitted = {0: 0, 1: 0}

    def take(events):
        nonlocal done_fit
        for (rid, model, kind, status, ts, t0, td, batch) in events:
            if kind == 1:
                srv.result(rid)
            if status != 0:
                continue
            lat[kind].append(td - ts)
            queue[kind].append(t0 - ts)
            service[kind].append(td - t0)
            if kind == 0:
                resident.append(model)
                done_fit += 1

    t_start = time.perf_counter()
    fi = pi = 0
    for t, kind in arrivals:
        while True:
            now = time.perf_counter() - t_start
            if now >= t:
                break
            take(srv.poll(timeout_s=min(t - now, 0.002)))
        if kind == 0:
            p = pool[fit_pick[fi]]
            fi += 1
            srv.submit_fit(p.X, p.y, p.c, p.lengthscale, 1.0)
            submitted[0] += 1
        else:
            m, q, u = int(pred_m[pi]), int(pred_q[pi]), float(pred_u[pi])
            pi += 1
            if not resident:
                skipped += 1
                continue
            try:
                srv.submit_predict(resident[int(u * len(resident))], qpool[q][:m])
                submitted[1] += 1
            except native.ItergpError:
                skipped += 1
    t_arr = time.perf_counter() - t_start
    t_end = t_arr + drain_s
    while time.perf_counter() - t_start < t_end and len(lat[0]) + len(lat[1]) < submitted[0] + submitted[1]:
        take(srv.poll(timeout_s=0.05))
    wall = time.perf_counter() - t_start
    st = srv.stats()
    srv.close()

    def pct(x, q):
        return float(np.percentile(np.asarray(x), q) * 1e3) if x else None

    def split(kind):   # where the latency goes: waiting for admission vs on the GPU
        return {"queue_p50_ms": pct(queue[kind], 50), "queue_p99_ms": pct(queue[kind], 99),
                "service_p50_ms": pct(service[kind], 50), "service_p99_ms": pct(service[kind], 99)}

    return {"precision": precision, "arrival_s": round(t_arr, 3), "wall_s": round(wall, 3),
            "fits": {"submitted": submitted[0], "done": len(lat[0]), "req_per_s": len(lat[0]) / wall,
                     "p50_ms": pct(lat[0], 50), "p99_ms": pct(lat[0], 99), **split(0)},
            "predicts": {"submitted": submitted[1], "done": len(lat[1]), "req_per_s": len(lat[1]) / wall,
                         "p50_ms": pct(lat[1], 50), "p99_ms": pct(lat[1], 99), **split(1),
                         "skipped_no_model": skipped},
            "backlog_at_end": {"fits": st["queued_fits"], "predicts": st["queued_predicts"]},
            "fit_batches": st["fit_batches"], "predict_batches": st["predict_batches"],
            "evicted": st["evicted"]}


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2310_20285_gb300 import datagen, native

    dev = torch.device("cuda", local)
    # rank r works on its own independent problem (weak scaling)
    X, y, Xs, ys, S = datagen.workload_kernel_bench(n=args.n, seed=replica_seed(rank))
    n = X.shape[0]
    tX = torch.as_tensor(X, device=dev)
    tS = torch.as_tensor(S, device=dev)
    Y = torch.empty((n, P), device=dev)

    def step(prec=args.precision):
        native.kmatvec(tX, tX, tS, kind="matern32", lengthscale=ELL, outputscale=OUT,
                       precision=prec, out=Y)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # autotune the launch variants of every product shape timed below (recorded in the
    # library's table, reported in the JSON line)
    tuning = []
    if not args.no_tune:
        shapes = [("kernel bench", 60000, D, P, "matern32", args.precision, False)]
        if rank == 0 and not args.no_extras:
            shapes += [("batched fits", 8192, 64, 16, "rbf", pr, True) for pr in ("bf16x3", "bf16_comp")]
            shapes += [("served mean + variance", 16384, 32, 128, "rbf", "bf16x3", True)]
            shapes += [("small-D product", 131072, 32, 16, "rbf", pr, False) for pr in ("bf16x3", "bf16_comp")]
        for label, tn, td, tp, kind, prec, items in shapes:
            vs, best = native.autotune(tn, td, tp, kind=kind, precision=prec, items=items,
                                       lengthscale=ELL if kind == "matern32" else 1.0)
            tuning.append({"shape": label, "n": tn, "d": td, "p": tp, "precision": prec,
                           "schedule": "items" if items else "single",
                           "variants_ms": {f"{e}w/{abs(st)}st{'/residentA' if st < 0 else ''}"
                                           f"{'/pair' if pr == 1 else '/pair192' if pr == 2 else ''}": round(ms, 4)
                                           for e, st, pr, ms in vs},
                           "chosen": (f"{best[0]} epilogue warps, {abs(best[1])} stages"
                                      f"{', resident A' if best[1] < 0 else ''}"
                                      f"{', CTA pairs' if best[2] == 1 else ''}"
                                      f"{', CTA pairs with 192-row chunks' if best[2] == 2 else ''}") if best else None})

    for _ in range(max(args.warmup, 3)):
        step()
    assert native.sync_status() == 0
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    native.timing_read()
    native.timing_enable(True)
    l0 = native.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    barrier()
    launches = native.launch_count() - l0
    native.timing_enable(False)
    kern_ms, kern_n = native.timing_read()
    clk = clocks.stop()
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    t_max = max_over_ranks(t_step, dist, dev)
    value = aggregate_rate(n * n, world, t_max)
    assert native.sync_status() == 0

    # ---- end to end through the C ABI with host buffers (copies in the timed region)
    hX = torch.as_tensor(X).pin_memory()
    hS = torch.as_tensor(S).pin_memory()
    hY = torch.empty((n, P), dtype=torch.float32).pin_memory()
    dX = torch.empty_like(tX)
    dS = torch.empty_like(tS)
    dY = torch.empty_like(Y)

    def e2e_step():
        dX.copy_(hX, non_blocking=True)
        dS.copy_(hS, non_blocking=True)
        native.kmatvec(dX, dX, dS, kind="matern32", lengthscale=ELL, outputscale=OUT,
                       precision=args.precision, out=dY)
        hY.copy_(dY, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 5))
    e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(e2e_steps):
        e2e_step()
    e1.record()
    barrier()
    t_e2e = e0.elapsed_time(e1) / 1e3 / e2e_steps
    # where an end-to-end step spends its time: one more (untimed) step with events between
    # its host-to-device copies, the product and the device-to-host copy
    seg = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    seg[0].record()
    dX.copy_(hX, non_blocking=True)
    dS.copy_(hS, non_blocking=True)
    seg[1].record()
    native.kmatvec(dX, dX, dS, kind="matern32", lengthscale=ELL, outputscale=OUT,
                   precision=args.precision, out=dY)
    seg[2].record()
    hY.copy_(dY, non_blocking=True)
    seg[3].record()
    seg[3].synchronize()
    h2d_ms, prod_ms, d2h_ms = (seg[i].elapsed_time(seg[i + 1]) for i in range(3))
    t_e2e = max_over_ranks(t_e2e, dist, dev)

    pk, pk_kind = peaks()
    prec = args.precision
    # what back-to-back tcgen05.mma get in the distance GEMM's shape, probed here: the wide
    # pair form's cta_group::2 SS MMAs of M = 256, N = 192 (16-bit operands); TF32 rows as
    # one CTA per SM, SS M = N = 128 (kind::tf32)
    mma_ceiling = native.probe_throughput("mma_ss_n128_tf32" if prec == "tf32" else "pair_mma_ss_n192_f16") / 1e12
    flops = 2.0 * n * n * (D + P)
    kernel_s = (kern_ms / max(kern_n, 1)) / 1e3
    achieved = flops / kernel_s / 1e12
    # MMA flops issued per algorithmic flop: split operands take three products per
    # contraction (distance over D, weighted sum over the points)
    d_terms = {"bf16x3": 3, "bf16_comp": 3, "bf16": 1, "tf32": 1}.get(prec, 1)
    p_terms = {"bf16x3": 3, "bf16_comp": 1, "bf16": 1, "tf32": 3}.get(prec, 1)
    issued = 2.0 * n * n * (D * d_terms + P * p_terms)
    # the peak of the dominant contraction's dtype: BF16 measured; TF32 = measured BF16 x the
    # nominal dense ratio 1.1 / 2.25; the FP32 form runs on the CUDA cores (probed FFMA)
    if prec == "fp32":
        peak, peak_kind, bound, kname = native.probe_throughput("ffma") / 1e12, "FP32 FFMA probed here", "alu", "kmv_simt_kernel"
    elif prec == "tf32":
        peak, peak_kind, bound, kname = pk["bf16_tflops"] * 1.1 / 2.25, f"{pk_kind} bf16 dense (burst) x 1.1/2.25 (tf32)", "tensor", "kmv_tc_kernel"
    else:
        peak, peak_kind, bound, kname = pk["bf16_tflops"], f"{pk_kind} bf16 dense (burst)", "tensor", "kmv_tc_kernel"
    # DRAM bytes per launch from the ncu capture of this kernel version (the wide pair form)
    # at N = 40000 (bf16x3, D = 784, P = 80: 962.1 MB read + 19.0 MB written), scaled by the
    # pairs processed (the lockstep schedule re-reads the B side once per wave, so traffic
    # grows like N^2)
    traffic = None
    if args.precision == "bf16x3":
        traffic = (962.06e6 + 19.03e6) * (n / 40000.0) ** 2
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at N=40000, "
                              "scaled by (N/40000)^2" if traffic else None,
            "algorithmic_bytes_per_launch": float(n * 832 * 4 + n * P * 4 * 2),
            "peak_kind": peak_kind,
            "kernel": kname, "kernel_ms": kernel_s * 1e3,
            "algorithmic_flops_per_launch": flops}
    if prec == "bf16x3":
        roof["frac_of_sustained"] = achieved / pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    if prec != "fp32":
        roof.update({"tensor_flops_issued_per_launch": issued, "mma_shape_ceiling_tflops": mma_ceiling,
                     "issued_frac_of_mma_shape_ceiling": issued / kernel_s / 1e12 / mma_ceiling})
        # the pair form's distance GEMM fed by its TMA ring (no epilogue), N = 128 vs 192:
        # why the product takes 192-row chunks
        roof["ring_fed_mma_tflops"] = {"pair_n128": native.probe_throughput("ring_pair_n128") / 1e12,
                                       "pair_n192": native.probe_throughput("ring_pair_n192") / 1e12}

    out = {"metric": METRIC, "value": value, "unit": "kernel-pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"bf16x3": "bf16x3 (FP16 hi/lo split operands with power-of-two scales, three MMA terms "
                               "per contraction, FP32 accumulate; FP32-accurate)",
                     "bf16_comp": "bf16_comp (FP16 hi/lo split distance, BF16 weighted sum, FP32 accumulate)",
                     "bf16": "bf16 (BF16 operands, FP32 accumulate)",
                     "tf32": "tf32 (TF32 distance operands, FP16 hi/lo split weighted sum, FP32 accumulate)",
                     "fp32": "f32"}[prec],
           "data": "synthetic",
           "config": {"workload": f"kernel product K(X,X)S, N={n}, D={D}, P={P}, Matern-3/2 l=28, s=1; "
                                  "784-D sparse clusters (19% non-zero), S ~ N(0,1)",
                      "precision": args.precision, "l2": "inputs exceed L2 (X is 188 MB FP32, 200 MB BF16 hi+lo)",
                      "parallelism": f"{world} independent problem(s), one per GPU"},
           "roofline": roof, "clocks": clk, "gpu_launches": int(launches), "tuning": tuning,
           "e2e": {"value": aggregate_rate(n * n, world, t_e2e), "unit": "kernel-pairs/s",
                   "h2d_bytes_per_step": int(hX.numel() * 4 + hS.numel() * 4),
                   "d2h_bytes_per_step": int(hY.numel() * 4), "ms_per_step": t_e2e * 1e3,
                   "breakdown_ms": {"h2d": h2d_ms, "product": prod_ms, "d2h": d2h_ms},
                   "h2d_gbs": (hX.numel() + hS.numel()) * 4 / (h2d_ms * 1e6),
                   "d2h_gbs": hY.numel() * 4 / (d2h_ms * 1e6)}}

    if rank == 0 and not args.no_extras:
        try:
            paths = {}
            for prec, k in (("bf16", 5), ("bf16_comp", 5), ("tf32", 5), ("fp32", 2)):
                step(prec)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(k):
                    step(prec)
                b.record()
                torch.cuda.synchronize()
                tp = a.elapsed_time(b) / 1e3 / k
                paths[prec] = {"kernel_pairs_per_s": n * n / tp, "ms": tp * 1e3}
            paths[args.precision] = {"kernel_pairs_per_s": n * n / t_step, "ms": t_step * 1e3}
            out["paths"] = paths
            # full IterNCGP fit on the same data: 5 Newton steps x <= 5 iterations, R = 200
            fits = {}
            ty = torch.as_tensor(y, device=dev)
            for prec in ("bf16x3", "bf16", "fp32"):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    m = native.fit(tX, ty, 10, kind="matern32", lengthscale=ELL, outputscale=OUT,
                                   precision=prec, max_newton=5, max_iters=5, rank=200)
                except native.ItergpError as e:
                    fits[prec] = {"error": str(e)}
                    continue
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                mean, var, probs = m.predict(torch.as_tensor(Xs, device=dev))
                acc = float((probs.argmax(1).cpu().numpy() == ys).mean())
                r = m.report
                fits[prec] = {"newton_step_ms": dt * 1e3 / max(r.newton_steps, 1),
                              "fit_s": dt, "iters": int(r.total_iters), "test_acc": acc,
                              "objective": [round(r.objective[i], 1) for i in range(r.newton_steps)]}
                m.free()
            out["fit"] = {"workload": "IterNCGP fit, same data, C=10, 5 Newton steps x 5 iterations, R=200",
                          "note": "the undamped Newton trajectory on this kernel (l = sqrt(D): K ~ 0.88 11^T) "
                                  "changes under product perturbations of 1e-7 relative (FP64 oracle with "
                                  "injected noise, N = 20000), so FP32/BF16 fits cannot follow it; times "
                                  "per Newton step are comparable, accuracies are not",
                          **fits}
        except Exception as e:   # noqa: BLE001 -- recorded in the line
            err = {"error": f"{type(e).__name__}: {str(e)[:300]}"}
            out.setdefault("paths", err)
            out.setdefault("fit", err)
    if rank == 0 and not args.no_extras:
        out["small_d_roofline"] = guarded(small_d_roofline, native, torch, dev)
        out["batched"] = guarded(bench_batched, native, datagen, torch, dev, args.batch_count)
    if rank == 0 and not args.no_extras:
        out["gmm_large"] = guarded(bench_gmm, native, datagen, torch, dev)
        out["class_kernels"] = guarded(bench_class_kernels, native, datagen, torch, dev)
        out["likelihoods"] = guarded(bench_likelihoods, native, datagen, torch, dev)
        out["poisson_study"] = guarded(bench_poisson_study, native, datagen, torch, dev)
    if rank == 0 and not args.no_extras and args.serve_seconds > 0:
        out["serving"] = {
            "workload": f"{args.serve_seconds:g} s of Poisson arrivals: fits 50/s (N log-U[1e3,5e4], D=32, C=5, "
                        "RBF l log-U[0.3,3], 5 Newton x <=5 iters, R=50) and predicts 2000/s (M U[1,4096], "
                        "D=32) against resident models; 80 GB model budget; latency = results in host "
                        "buffers minus submission",
            "forms": [guarded(bench_serving, native, datagen, prec, args.serve_seconds)
                      for prec in ("bf16x3", "fp32")]}
    if rank == 0 and not args.no_extras:
        out["newton_step_small"] = guarded(newton_step_ms_small, native, datagen, torch, dev)
    if rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(X, S, args.cpu_seconds)
        out["cpu_baseline"]["one_core"] = cpu_baseline_one_core(X.shape[0], min(5.0, args.cpu_seconds / 3))
        if not args.no_extras:
            runs = guarded(cpu_baseline_oracle_runs, native, datagen, torch, dev, X, S, min(10.0, args.cpu_seconds))
            if isinstance(runs, dict) and "accuracy" in runs:
                out["accuracy"] = runs.pop("accuracy")
            out["cpu_baseline"]["oracle_runs"] = runs
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
