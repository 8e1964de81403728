"""The C-ABI library loads and exports every symbol include/itergp.h declares; host-side
argument validation rejects bad input before any launch (no GPU needed)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "itergp.h")
LIB = os.path.join(ROOT, "paper_2310_20285_gb300", "libitergp.so")


def declared_functions(header=HEADER):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(itergp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2310_20285_gb300 import build
        build.build()
    return ct.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("itergp_fit", "itergp_kmatvec", "itergp_predict", "itergp_model_free",
                     "itergp_status_string"):
        assert required in names


def header_enum_values():
    """NAME = value pairs of every enumerator in the header."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ITERGP_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_constants_match_the_header(lib):
    """The Python binding's codes for precisions, kernels, likelihoods and policies are the
    header's enumerators (the binding is loaded on the host only; no CUDA call is made)."""
    from paper_2310_20285_gb300 import native
    h = header_enum_values()
    assert native.PRECISIONS == {"fp32": h["ITERGP_FP32"], "bf16x3": h["ITERGP_BF16X3"], "bf16": h["ITERGP_BF16"],
                                 "bf16_comp": h["ITERGP_BF16_COMP"], "tf32": h["ITERGP_TF32"]}
    assert native.KERNELS == {"rbf": h["ITERGP_RBF"], "matern32": h["ITERGP_MATERN32"]}
    assert native.LIKELIHOODS == {"softmax": h["ITERGP_LIK_SOFTMAX"], "bernoulli": h["ITERGP_LIK_BERNOULLI"],
                                  "poisson": h["ITERGP_LIK_POISSON"], "gaussian": h["ITERGP_LIK_GAUSSIAN"]}
    assert (native.POLICY_CG, native.POLICY_UNIT) == (h["ITERGP_POLICY_CG"], h["ITERGP_POLICY_UNIT"])
    assert native.TUNE_MAX == int(re.search(r"#define ITERGP_TUNE_MAX (\d+)", open(HEADER).read()).group(1))


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_probe_library_is_separate_and_exports_its_header():
    """The bench's throughput probes live in their own library, not in the product's."""
    probe_h = os.path.join(ROOT, "include", "itergp_probe.h")
    probe_so = os.path.join(ROOT, "paper_2310_20285_gb300", "libitergp_probe.so")
    if not os.path.exists(probe_so):
        from paper_2310_20285_gb300 import build
        build.build()
    names = declared_functions(probe_h)
    assert names == ["itergp_probe_throughput"]
    plib = ct.CDLL(probe_so)
    assert all(hasattr(plib, n) for n in names)
    assert not hasattr(ct.CDLL(LIB), "itergp_probe_throughput")


def test_status_strings(lib):
    lib.itergp_status_string.restype = ct.c_char_p
    lib.itergp_status_string.argtypes = [ct.c_int]
    assert lib.itergp_status_string(0) == b"ok"
    assert b"bound" in lib.itergp_status_string(-5)
    assert lib.itergp_status_string(12345) == b"unknown status"


class Kernel(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("lengthscale", ct.c_float), ("outputscale", ct.c_float)]


@pytest.mark.parametrize("kind,ell,s,prec,m,n,d,p", [
    (7, 1.0, 1.0, 0, 4, 4, 2, 1),      # unknown kernel
    (0, 0.0, 1.0, 0, 4, 4, 2, 1),      # zero lengthscale
    (0, 1.0, -1.0, 0, 4, 4, 2, 1),     # negative outputscale
    (0, 1.0, 1.0, 9, 4, 4, 2, 1),      # unknown precision
    (0, 1.0, 1.0, 5, 4, 4, 2, 1),      # the first code past ITERGP_TF32
    (0, 1.0, 1.0, -1, 4, 4, 2, 1),     # negative precision
    (0, 1.0, 1.0, 0, -1, 4, 2, 1),     # negative m
    (0, 1.0, 1.0, 0, 4, 4, 0, 1),      # d = 0
    (0, 1.0, 1.0, 0, 4, 4, 5000, 1),   # d too large
])
def test_kmatvec_rejects_bad_arguments_on_the_host(lib, kind, ell, s, prec, m, n, d, p):
    k = Kernel(kind, ell, s)
    f = lib.itergp_kmatvec
    f.restype = ct.c_int
    f.argtypes = [ct.POINTER(Kernel), ct.c_int32, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int64,
                  ct.c_int64, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p]
    dummy = ct.c_void_p(16)
    assert f(ct.byref(k), prec, dummy, m, dummy, n, d, dummy, p, dummy, None) == -1


def test_kmatvec_null_output_rejected(lib):
    k = Kernel(0, 1.0, 1.0)
    f = lib.itergp_kmatvec
    f.restype = ct.c_int
    f.argtypes = [ct.POINTER(Kernel), ct.c_int32, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int64,
                  ct.c_int64, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p]
    dummy = ct.c_void_p(16)
    assert f(ct.byref(k), 0, dummy, 4, dummy, 4, 2, dummy, 3, None, None) == -1


def test_fit_rejects_bad_arguments_on_the_host(lib):
    from paper_2310_20285_gb300.native import FitParams, FitReport, Kernel as K
    f = lib.itergp_fit
    f.restype = ct.c_int
    f.argtypes = [ct.POINTER(FitParams), ct.POINTER(ct.c_void_p), ct.POINTER(FitReport), ct.c_void_p]
    base = dict(n=10, d=2, c=3, X=16, y=16, kernel=K(0, 1.0, 1.0), precision=0, policy=0,
                max_newton=1, max_iters=1, rank=-1, recycle=1, literal_kv=0, tol_newton=0.0,
                tol_abs=1e-5, tol_rel=1e-5)
    for bad in (dict(n=0), dict(c=1), dict(c=65), dict(d=0), dict(X=None), dict(y=None),
                dict(policy=5), dict(max_newton=0), dict(max_iters=-1), dict(precision=8),
                dict(kernel=K(0, -1.0, 1.0)), dict(tol_abs=-1.0),
                dict(wait_limit_ns=999), dict(wait_limit_ns=10 ** 11)):   # outside 1e6 .. 6e10 ns
        prm = FitParams(**{**base, **bad})
        h = ct.c_void_p()
        assert f(ct.byref(prm), ct.byref(h), None, None) == -1, bad
        assert not h.value
    assert f(None, None, None, None) == -1


def test_predict_rejects_null_model(lib):
    f = lib.itergp_predict
    f.restype = ct.c_int
    f.argtypes = [ct.c_void_p] * 7
    assert f(None, ct.c_void_p(16), 3, ct.c_void_p(16), None, None, None) == -1


def test_model_free_accepts_null(lib):
    lib.itergp_model_free.argtypes = [ct.c_void_p]
    lib.itergp_model_free.restype = None
    lib.itergp_model_free(None)


class ServerConfig(ct.Structure):
    _fields_ = [("model_bytes", ct.c_int64), ("work_bytes", ct.c_int64), ("kind", ct.c_int32),
                ("precision", ct.c_int32), ("d_max", ct.c_int32), ("c_max", ct.c_int32),
                ("max_fit_batch", ct.c_int32), ("max_predict_batch", ct.c_int32),
                ("max_predict_rows", ct.c_int64), ("max_newton", ct.c_int32),
                ("max_iters", ct.c_int32), ("rank", ct.c_int32), ("graph", ct.c_int32),
                ("tol_abs", ct.c_double), ("tol_rel", ct.c_double)]


def test_server_config_is_validated_on_the_host(lib):
    """Invalid server configurations fail with EINVAL before any CUDA call (no GPU here)."""
    lib.itergp_server_create.argtypes = [ct.POINTER(ServerConfig), ct.POINTER(ct.c_void_p)]
    lib.itergp_server_create.restype = ct.c_int

    def cfg(**kw):
        base = dict(model_bytes=1 << 30, work_bytes=1 << 30, kind=0, precision=0, d_max=32, c_max=5,
                    max_fit_batch=8, max_predict_batch=8, max_predict_rows=1 << 16, max_newton=5,
                    max_iters=5, rank=50, graph=1, tol_abs=1e-5, tol_rel=1e-5)
        base.update(kw)
        return ServerConfig(**base)

    h = ct.c_void_p()
    for bad in (dict(model_bytes=0), dict(d_max=0), dict(c_max=1), dict(c_max=17), dict(kind=7),
                dict(precision=9), dict(max_fit_batch=0), dict(max_predict_rows=100),
                dict(max_iters=0), dict(tol_abs=-1.0),
                dict(c_max=6)):   # 6 classes x 25 buffer columns > 128 variance weight rows
        assert lib.itergp_server_create(ct.byref(cfg(**bad)), ct.byref(h)) == -1, bad
        assert not h.value


def test_tune_cache_round_trip(lib, tmp_path):
    """The variant table's text cache loads, merges and saves without a GPU; malformed
    lines are rejected."""
    lib.itergp_tune_load.argtypes = [ct.c_char_p]
    lib.itergp_tune_save.argtypes = [ct.c_char_p]
    src = tmp_path / "in.txt"
    src.write_text("# comment\n1 0 64 16 1 8 2\n3 1 832 80 0 4 0 0\n2 0 64 16 1 4 5 1\n"
                   "1 1 832 80 0 8 3 0 1\n4 0 832 80 0 4 3 0 2\n")
    assert lib.itergp_tune_clear() == 0
    assert lib.itergp_tune_load(str(src).encode()) == 0
    out = tmp_path / "out.txt"
    assert lib.itergp_tune_save(str(out).encode()) == 0
    rows = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    # missing resident-A / CTA-pair columns read as -1 (automatic)
    assert sorted(rows) == sorted(["1 0 64 16 1 8 2 -1 -1", "3 1 832 80 0 4 0 0 -1", "2 0 64 16 1 4 5 1 -1",
                                   "1 1 832 80 0 8 3 0 1", "4 0 832 80 0 4 3 0 2"])
    bad = tmp_path / "bad.txt"
    bad.write_text("1 0 64 16 1 6 2\n")          # 6 epilogue warps is not a variant
    assert lib.itergp_tune_load(str(bad).encode()) == -1
    bad.write_text("1 0 64 16 1 8 2 0 3\n")      # the pair column takes -1, 0, 1 or 2 (wide chunks)
    assert lib.itergp_tune_load(str(bad).encode()) == -1
    assert lib.itergp_tune_clear() == 0


def test_throughput_probe_rejects_bad_arguments():
    """Unknown probes and a null result pointer fail with EINVAL before any CUDA call."""
    f = ct.CDLL(os.path.join(ROOT, "paper_2310_20285_gb300", "libitergp_probe.so")).itergp_probe_throughput
    f.restype = ct.c_int
    f.argtypes = [ct.c_int32, ct.POINTER(ct.c_double), ct.c_void_p]
    out = ct.c_double()
    for what in (-1, 15, 99):
        assert f(what, ct.byref(out), None) == -1
    assert f(0, None, None) == -1


def test_class_kernel_product_rejects_bad_arguments(lib):
    """itergp_kmatvec_classes validates its kernel list and sizes before any CUDA call."""
    class K(ct.Structure):
        _fields_ = [("kind", ct.c_int32), ("lengthscale", ct.c_float), ("outputscale", ct.c_float)]
    f = lib.itergp_kmatvec_classes
    f.restype = ct.c_int
    f.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_int64,
                  ct.c_int64, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p]
    good = (K * 3)(K(0, 1.0, 1.0), K(1, 2.0, 0.5), K(0, 0.5, 2.0))
    bad = (K * 3)(K(0, 1.0, 1.0), K(1, -2.0, 0.5), K(0, 0.5, 2.0))
    p = ct.c_void_p(16)
    assert f(None, 3, 0, p, 10, p, 10, 2, p, 3, p, None) == -1          # no kernels
    assert f(good, 0, 0, p, 10, p, 10, 2, p, 3, p, None) == -1          # c < 1
    assert f(good, 65, 0, p, 10, p, 10, 2, p, 3, p, None) == -1         # c > 64
    assert f(bad, 3, 0, p, 10, p, 10, 2, p, 3, p, None) == -1           # a bad lengthscale
    assert f(good, 3, 9, p, 10, p, 10, 2, p, 3, p, None) == -1          # unknown precision
    assert f(good, 3, 0, p, 10, p, 10, 0, p, 3, p, None) == -1          # d < 1
    assert f(good, 3, 0, p, 10, p, 10, 2, p, 3, None, None) == -1       # no output
