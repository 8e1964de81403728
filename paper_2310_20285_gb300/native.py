"""ctypes binding of libitergp (the C ABI declared in include/itergp.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  PyTorch provides device memory and the current CUDA stream.  If the shared
library is missing this module raises at import; there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libitergp.so")

OK, EINVAL, ENOMEM, ECUDA, ENUMERIC, ETIMEOUT, EUNSUPPORTED, ESCRATCH, EGONE = 0, -1, -2, -3, -4, -5, -6, -7, -8
NOALLOC_SCRATCH_BYTES = 64 << 20
RBF, MATERN32 = 0, 1
FP32, BF16X3, BF16, BF16_COMP, TF32 = 0, 1, 2, 3, 4
POLICY_CG, POLICY_UNIT = 0, 1
STOP_MAXITER, STOP_TOL, STOP_ETA = 0, 1, 2
MAX_REPORT_STEPS = 64

PRECISIONS = {"fp32": FP32, "bf16x3": BF16X3, "bf16": BF16, "bf16_comp": BF16_COMP, "tf32": TF32}
LIKELIHOODS = {"softmax": 0, "bernoulli": 1, "poisson": 2, "gaussian": 3}
KERNELS = {"rbf": RBF, "matern32": MATERN32}


class ItergpError(RuntimeError):
    """A non-zero status of a library call; `code` is the itergp_status value."""

    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_string(code)} ({code})")
        self.code = code


class Kernel(ct.Structure):
    """itergp_kernel: kind (RBF or MATERN32), lengthscale l, outputscale s."""
    _fields_ = [("kind", ct.c_int32), ("lengthscale", ct.c_float), ("outputscale", ct.c_float)]


class FitParams(ct.Structure):
    """itergp_fit_params (field order and types as in include/itergp.h)."""
    _fields_ = [("n", ct.c_int64), ("d", ct.c_int64), ("c", ct.c_int32),
                ("X", ct.c_void_p), ("y", ct.c_void_p), ("kernel", Kernel),
                ("precision", ct.c_int32), ("policy", ct.c_int32),
                ("max_newton", ct.c_int32), ("max_iters", ct.c_int32), ("rank", ct.c_int32),
                ("recycle", ct.c_int32), ("literal_kv", ct.c_int32),
                ("tol_newton", ct.c_double), ("tol_abs", ct.c_double), ("tol_rel", ct.c_double),
                ("graph", ct.c_int32), ("f0", ct.c_void_p), ("likelihood", ct.c_int32),
                ("noise", ct.c_float), ("y_real", ct.c_void_p),
                ("class_kernels", ct.POINTER(Kernel)), ("wait_limit_ns", ct.c_uint64)]


class FitReport(ct.Structure):
    """itergp_fit_report: per Newton step iterations, stop reasons, kept buffer columns,
    objective and relative change; final residual norm, the model's device bytes and the
    call's peak pool bytes."""
    _fields_ = [("newton_steps", ct.c_int32), ("total_iters", ct.c_int32),
                ("buffer_cols", ct.c_int32), ("stop_reason", ct.c_int32),
                ("iters", ct.c_int32 * MAX_REPORT_STEPS), ("stops", ct.c_int32 * MAX_REPORT_STEPS),
                ("kept", ct.c_int32 * MAX_REPORT_STEPS),
                ("objective", ct.c_double * MAX_REPORT_STEPS),
                ("rel_change", ct.c_double * MAX_REPORT_STEPS),
                ("resid_norm", ct.c_double), ("device_bytes", ct.c_int64),
                ("status", ct.c_int32), ("reserved", ct.c_int32), ("peak_bytes", ct.c_int64)]


class ModelView(ct.Structure):
    """itergp_model_view: sizes and device pointers of a model's X, v, f and Q."""
    _fields_ = [("n", ct.c_int64), ("d", ct.c_int64), ("c", ct.c_int32),
                ("buffer_cols", ct.c_int32), ("kernel", Kernel),
                ("X", ct.c_void_p), ("v", ct.c_void_p), ("f", ct.c_void_p), ("Q", ct.c_void_p)]


class ServerConfig(ct.Structure):
    """itergp_server_config: memory budgets, shared kernel kind, precision and schedule."""
    _fields_ = [("model_bytes", ct.c_int64), ("work_bytes", ct.c_int64), ("kind", ct.c_int32),
                ("precision", ct.c_int32), ("d_max", ct.c_int32), ("c_max", ct.c_int32),
                ("max_fit_batch", ct.c_int32), ("max_predict_batch", ct.c_int32),
                ("max_predict_rows", ct.c_int64), ("max_newton", ct.c_int32),
                ("max_iters", ct.c_int32), ("rank", ct.c_int32), ("graph", ct.c_int32),
                ("tol_abs", ct.c_double), ("tol_rel", ct.c_double)]


class ServerEvent(ct.Structure):
    """itergp_server_event: one completed request with its submit, start and done times."""
    _fields_ = [("id", ct.c_int64), ("model", ct.c_int64), ("kind", ct.c_int32),
                ("status", ct.c_int32), ("submit_s", ct.c_double), ("start_s", ct.c_double),
                ("done_s", ct.c_double), ("batch", ct.c_int32), ("reserved", ct.c_int32)]


class ServerStats(ct.Structure):
    """itergp_server_stats: resident models and rows, completed work and queue lengths."""
    _fields_ = [(n, ct.c_int64) for n in ("resident_models", "resident_rows", "slab_rows",
                                          "fits_done", "predicts_done", "fit_batches",
                                          "predict_batches", "evicted", "queued_fits",
                                          "queued_predicts")]


REQ_FIT, REQ_PREDICT = 0, 1
TUNE_MAX = 20


class TuneVariant(ct.Structure):
    """One timed launch variant: epilogue warps, ring stages (< 0: resident A), CTA-pair
    form (1) or one CTA per tile (0), ms."""
    _fields_ = [("epilogue_warps", ct.c_int32), ("stages", ct.c_int32), ("cta_pair", ct.c_int32),
                ("ms", ct.c_double)]


class TuneResult(ct.Structure):
    """itergp_tune_result: up to TUNE_MAX timed variants and the index of the fastest."""
    _fields_ = [("count", ct.c_int32), ("best", ct.c_int32), ("variants", TuneVariant * TUNE_MAX)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libitergp.so not built ({_LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(_LIB_PATH)
    vp, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int32
    lib.itergp_kmatvec.argtypes = [ct.POINTER(Kernel), i32, vp, i64, vp, i64, i64, vp, i64, vp, vp]
    lib.itergp_kmatvec_classes.argtypes = [ct.POINTER(Kernel), i32, i32, vp, i64, vp, i64, i64, vp, i64,
                                           vp, vp]
    lib.itergp_kmatvec_noalloc.argtypes = [ct.POINTER(Kernel), i32, vp, i64, vp, i64, i64, vp, i64,
                                           vp, vp, vp]
    lib.itergp_winv_apply.argtypes = [vp, i64, i32, vp, vp, vp]
    lib.itergp_pseudo_targets.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.itergp_sym_eig.argtypes = [vp, i32, vp, vp, vp]
    lib.itergp_fit.argtypes = [ct.POINTER(FitParams), ct.POINTER(vp), ct.POINTER(FitReport), vp]
    lib.itergp_fit_batch.argtypes = [ct.POINTER(FitParams), i32, ct.POINTER(vp), ct.POINTER(FitReport), vp]
    lib.itergp_predict.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    lib.itergp_model_get_view.argtypes = [vp, ct.POINTER(ModelView)]
    lib.itergp_model_free.argtypes = [vp]
    lib.itergp_model_free.restype = None
    lib.itergp_sync_status.argtypes = [vp]
    lib.itergp_status_string.argtypes = [i32]
    lib.itergp_status_string.restype = ct.c_char_p
    lib.itergp_version.restype = ct.c_char_p
    lib.itergp_last_error.restype = ct.c_char_p
    lib.itergp_last_error.argtypes = []
    lib.itergp_timing_enable.argtypes = [ct.c_int]
    lib.itergp_timing_read.argtypes = [ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)]
    lib.itergp_launch_count.restype = ct.c_int64
    lib.itergp_launch_count.argtypes = []
    lib.itergp_server_create.argtypes = [ct.POINTER(ServerConfig), ct.POINTER(vp)]
    lib.itergp_server_destroy.argtypes = [vp]
    lib.itergp_server_submit_fit.argtypes = [vp, vp, vp, i64, i64, i32, ct.c_float, ct.c_float,
                                             ct.POINTER(i64)]
    lib.itergp_server_submit_predict.argtypes = [vp, i64, vp, i64, vp, vp, vp, ct.POINTER(i64)]
    lib.itergp_server_poll.argtypes = [vp, ct.POINTER(ServerEvent), i32, ct.POINTER(i32), i64]
    lib.itergp_server_release.argtypes = [vp, i64]
    lib.itergp_server_get_stats.argtypes = [vp, ct.POINTER(ServerStats)]
    lib.itergp_autotune.argtypes = [ct.POINTER(Kernel), i32, i64, i64, i64, i32, ct.POINTER(TuneResult), vp]
    lib.itergp_tune_save.argtypes = [ct.c_char_p]
    lib.itergp_tune_load.argtypes = [ct.c_char_p]
    lib.itergp_tune_clear.argtypes = []
    lib.itergp_selftest_wait.argtypes = [ct.c_uint64, vp]
    lib.itergp_selftest_wait.restype = ct.c_int
    for name in ("itergp_autotune", "itergp_tune_save", "itergp_tune_load", "itergp_tune_clear",
                 "itergp_kmatvec", "itergp_kmatvec_noalloc", "itergp_winv_apply", "itergp_pseudo_targets",
                 "itergp_sym_eig", "itergp_fit", "itergp_fit_batch", "itergp_predict",
                 "itergp_model_get_view", "itergp_sync_status", "itergp_server_create",
                 "itergp_server_destroy", "itergp_server_submit_fit", "itergp_server_submit_predict",
                 "itergp_server_poll", "itergp_server_release", "itergp_server_get_stats"):
        getattr(lib, name).restype = ct.c_int
    return lib


lib = _load()


def status_string(code: int) -> str:
    """The library's text for an itergp_status code."""
    return lib.itergp_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != OK:
        detail = lib.itergp_last_error().decode() if code == ECUDA else ""
        raise ItergpError(code, f"{where} [{detail}]" if detail else where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return ct.c_void_p(t.data_ptr())


def _kernel(kind, lengthscale, outputscale) -> Kernel:
    k = KERNELS[kind] if isinstance(kind, str) else int(kind)
    return Kernel(k, float(lengthscale), float(outputscale))


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def kmatvec(A, B, S, kind="rbf", lengthscale=1.0, outputscale=1.0, precision="fp32",
            out=None, stream=None):
    """Y = k(A, B) @ S on the GPU, k never stored.  A: m x d, B: n x d, S: n x p (float32)."""
    m, d = A.shape
    n = B.shape[0]
    p = S.shape[1]
    if out is None:
        out = torch.empty((m, p), device=A.device, dtype=torch.float32)
    k = _kernel(kind, lengthscale, outputscale)
    rc = lib.itergp_kmatvec(ct.byref(k), _prec(precision), _dev(A, torch.float32, "A"), m,
                            _dev(B, torch.float32, "B"), n, d, _dev(S, torch.float32, "S"), p,
                            _dev(out, torch.float32, "out"), _stream(stream))
    _check(rc, "itergp_kmatvec")
    return out


def _class_kernels(kernels):
    """[(kind, lengthscale, outputscale), ...] -> a ctypes array of itergp_kernel."""
    arr = (Kernel * len(kernels))()
    for i, (kind, ell, s) in enumerate(kernels):
        arr[i] = _kernel(kind, ell, s)
    return arr


def kmatvec_classes(A, B, S, kernels, precision="fp32", out=None, stream=None):
    """Y[:, j] = k_{j mod c}(A, B) @ S[:, j] with one kernel per class (c = len(kernels);
    the columns of S are n x c blocks side by side, CN ordering)."""
    m, d = A.shape
    n = B.shape[0]
    p = S.shape[1]
    if out is None:
        out = torch.empty((m, p), device=A.device, dtype=torch.float32)
    ks = _class_kernels(kernels)
    rc = lib.itergp_kmatvec_classes(ks, len(kernels), _prec(precision), _dev(A, torch.float32, "A"), m,
                                    _dev(B, torch.float32, "B"), n, d, _dev(S, torch.float32, "S"), p,
                                    _dev(out, torch.float32, "out"), _stream(stream))
    _check(rc, "itergp_kmatvec_classes")
    return out


def kmatvec_noalloc(A, B, S, kind="rbf", lengthscale=1.0, outputscale=1.0, precision="fp32",
                    out=None, status=None, stream=None):
    """Same product as kmatvec, computed without any device allocation by the library (its
    scratch is a fixed static device array; see itergp_kmatvec_noalloc).  ``out`` and the
    optional int32 ``status`` word are the caller's."""
    m, d = A.shape
    n = B.shape[0]
    p = S.shape[1]
    if out is None:
        out = torch.empty((m, p), device=A.device, dtype=torch.float32)
    k = _kernel(kind, lengthscale, outputscale)
    st = None if status is None else _dev(status, torch.int32, "status")
    rc = lib.itergp_kmatvec_noalloc(ct.byref(k), _prec(precision), _dev(A, torch.float32, "A"), m,
                                    _dev(B, torch.float32, "B"), n, d, _dev(S, torch.float32, "S"),
                                    p, _dev(out, torch.float32, "out"), st, _stream(stream))
    _check(rc, "itergp_kmatvec_noalloc")
    return out


def winv_apply(f, x, out=None, stream=None):
    """W^+ x for the softmax likelihood at f (Lemma A.6): per point P diag(1/pi) P x."""
    n, c = f.shape
    out = torch.empty_like(x) if out is None else out
    _check(lib.itergp_winv_apply(_dev(f, torch.float32, "f"), n, c, _dev(x, torch.float32, "x"),
                                 _dev(out, torch.float32, "out"), _stream(stream)), "itergp_winv_apply")
    return out


def pseudo_targets(f, y, out=None, stream=None):
    """y_hat = f + W^+ grad log p(y|f) for the softmax likelihood (Alg. 1)."""
    n, c = f.shape
    out = torch.empty_like(f) if out is None else out
    _check(lib.itergp_pseudo_targets(_dev(f, torch.float32, "f"), _dev(y, torch.int32, "y"), n, c,
                                     _dev(out, torch.float32, "out"), _stream(stream)),
           "itergp_pseudo_targets")
    return out


def sym_eig(M, stream=None):
    """Eigenvalues (descending) and eigenvectors of a symmetric FP64 matrix on the GPU
    (the Jacobi solver of Alg. 3's virtual solver run)."""
    b = M.shape[0]
    lam = torch.empty(b, device=M.device, dtype=torch.float64)
    U = torch.empty((b, b), device=M.device, dtype=torch.float64)
    _check(lib.itergp_sym_eig(_dev(M, torch.float64, "M"), b, _dev(lam, torch.float64, "lam"),
                              _dev(U, torch.float64, "U"), _stream(stream)), "itergp_sym_eig")
    return lam, U


def timing_enable(on: bool = True):
    """Bracket every fused kernel-product launch with CUDA events on its stream."""
    lib.itergp_timing_enable(1 if on else 0)


def timing_read():
    """(summed device ms, number of fused kernel-product launches) since the last read."""
    ms, n = ct.c_double(), ct.c_int64()
    _check(lib.itergp_timing_read(ct.byref(ms), ct.byref(n)), "itergp_timing_read")
    return ms.value, n.value


def launch_count() -> int:
    """Total kernels the library has launched in this process."""
    return int(lib.itergp_launch_count())


def sync_status(stream=None) -> int:
    """Wait for the stream, then read and clear the device status word (0: no error)."""
    return int(lib.itergp_sync_status(_stream(stream)))


class Model:
    """A fitted IterNCGP model living in device memory (owned by the library)."""

    def __init__(self, handle: ct.c_void_p, report: FitReport, device):
        self._h = handle
        self.report = report
        self.device = device

    def view(self) -> ModelView:
        """Sizes and device pointers of the model's arrays (owned by the model)."""
        v = ModelView()
        _check(lib.itergp_model_get_view(self._h, ct.byref(v)), "itergp_model_get_view")
        return v

    def _wrap(self, ptr, shape):
        """Copy a device array owned by the model into a new torch tensor."""
        if any(x == 0 for x in shape):
            return torch.empty(shape, device=self.device, dtype=torch.float32)
        view = torch.as_tensor(_CudaArray(ptr, shape), device=self.device)
        return view.clone()

    def arrays(self):
        """Copies of v (n x c), f (n x c) and the root Q (buffer columns x n x c)."""
        v = self.view()
        n, c, B = v.n, v.c, v.buffer_cols
        return {"v": self._wrap(v.v, (n, c)), "f": self._wrap(v.f, (n, c)),
                "Q": self._wrap(v.Q, (B, n, c))}

    def predict(self, Xs, want_var=True, want_probs=True, stream=None):
        """Predictive mean, marginal variance and the likelihood's third output (class
        probabilities by the probit approximation for softmax and Bernoulli, E[e^f] for
        Poisson, the mean for Gaussian) at the rows of Xs (Eqs. 9-10)."""
        m = Xs.shape[0]
        c = self.view().c
        mean = torch.empty((m, c), device=Xs.device, dtype=torch.float32)
        var = torch.empty_like(mean) if want_var else None
        probs = torch.empty_like(mean) if want_probs else None
        rc = lib.itergp_predict(self._h, _dev(Xs, torch.float32, "Xs"), m,
                                _dev(mean, torch.float32, "mean"),
                                None if var is None else _dev(var, torch.float32, "var"),
                                None if probs is None else _dev(probs, torch.float32, "probs"),
                                _stream(stream))
        _check(rc, "itergp_predict")
        return mean, var, probs

    def free(self):
        """Release the model's device memory (idempotent)."""
        if self._h:
            lib.itergp_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for a float32 device array."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": "<f4",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _params(X, y, c, kind, lengthscale, outputscale, precision, policy, max_newton, max_iters,
            rank, recycle, literal_kv, tol_newton, tol_abs, tol_rel, graph, f0=None,
            likelihood="softmax", noise=1.0, class_kernels=None, wait_limit_ns=0) -> FitParams:
    n, d = X.shape
    prm = FitParams()
    prm.wait_limit_ns = int(wait_limit_ns)
    prm.n, prm.d, prm.c = n, d, int(c)
    prm.X = _dev(X, torch.float32, "X").value
    prm.likelihood = LIKELIHOODS[likelihood]
    if likelihood == "gaussian":   # real targets, n x c
        if y.numel() != n * int(c):
            raise ValueError("gaussian targets must be n x c")
        prm.y_real = _dev(y, torch.float32, "y").value
        prm.noise = float(noise)
    else:
        prm.y = _dev(y, torch.int32, "y").value
    prm.kernel = _kernel(kind, lengthscale, outputscale)
    prm.precision = _prec(precision)
    prm.policy = POLICY_CG if policy in ("cg", POLICY_CG) else POLICY_UNIT
    prm.max_newton, prm.max_iters = int(max_newton), int(max_iters)
    prm.rank = -1 if rank is None else int(rank)
    prm.recycle, prm.literal_kv = int(bool(recycle)), int(bool(literal_kv))
    prm.tol_newton, prm.tol_abs, prm.tol_rel = float(tol_newton), float(tol_abs), float(tol_rel)
    prm.graph = int(bool(graph))
    if f0 is not None:
        if tuple(f0.shape) != (n, int(c)):
            raise ValueError("f0 must be n x c")
        prm.f0 = _dev(f0, torch.float32, "f0").value
    if class_kernels is not None:
        if len(class_kernels) != int(c):
            raise ValueError("one kernel per class expected")
        prm._class_kernels = _class_kernels(class_kernels)   # kept alive with the params
        prm.class_kernels = prm._class_kernels
    return prm


def fit(X, y, c, kind="rbf", lengthscale=1.0, outputscale=1.0, precision="fp32",
        policy="cg", max_newton=10, max_iters=50, rank=-1, recycle=True, literal_kv=False,
        tol_newton=0.0, tol_abs=1e-5, tol_rel=1e-5, graph=False, stream=None, f0=None,
        likelihood="softmax", noise=1.0, class_kernels=None, wait_limit_ns=0) -> Model:
    """IterNCGP fit (Alg. 1-3) on the GPU.  likelihood: "softmax" (c >= 2 classes, integer
    labels), "bernoulli" (c = 1, labels 0/1), "poisson" (c = 1, counts) or "gaussian"
    (real targets y of n x c, noise variance `noise`).  f0 (n x c, device) starts Newton's
    method at that iterate instead of m = 0.  class_kernels: [(kind, lengthscale,
    outputscale)] * c gives each output GP its own kernel (then kind / lengthscale /
    outputscale are unused).  wait_limit_ns bounds every device-side wait of the fit's
    kernel products (0: the default 4 s)."""
    prm = _params(X, y, c, kind, lengthscale, outputscale, precision, policy, max_newton,
                  max_iters, rank, recycle, literal_kv, tol_newton, tol_abs, tol_rel, graph, f0,
                  likelihood, noise, class_kernels, wait_limit_ns)
    h = ct.c_void_p()
    rep = FitReport()
    rc = lib.itergp_fit(ct.byref(prm), ct.byref(h), ct.byref(rep), _stream(stream))
    _check(rc, "itergp_fit")
    return Model(h, rep, X.device)


def fit_batch(problems, kind="rbf", precision="fp32", policy="cg", max_newton=5, max_iters=5,
              rank=50, recycle=True, tol_newton=0.0, tol_abs=1e-5, tol_rel=1e-5, graph=True,
              stream=None, errors="raise"):
    """Batched fit of independent problems [(X, y, c, lengthscale, outputscale), ...] with
    one schedule (one launch per phase over all problems).  Returns a list of Models.  A
    problem that fails on the device fails alone: errors="raise" frees the other models
    and raises its ItergpError; errors="return" puts the ItergpError in its slot."""
    prms = (FitParams * len(problems))()
    keep = []
    for i, prob in enumerate(problems):   # an optional 6th entry: [(kind, l, s)] * c per class
        X, y, c, ell, s = prob[:5]
        ck = prob[5] if len(prob) > 5 else None
        pi = _params(X, y, c, kind, ell, s, precision, policy, max_newton, max_iters, rank,
                     recycle, False, tol_newton, tol_abs, tol_rel, graph, class_kernels=ck)
        keep.append(pi)
        prms[i] = pi
    hs = (ct.c_void_p * len(problems))()
    reps = (FitReport * len(problems))()
    rc = lib.itergp_fit_batch(prms, len(problems), hs, reps, _stream(stream))
    _check(rc, "itergp_fit_batch")
    out = [Model(ct.c_void_p(hs[i]), reps[i], problems[i][0].device) if hs[i]
           else ItergpError(reps[i].status, f"itergp_fit_batch (problem {i})")
           for i in range(len(problems))]
    failed = [o for o in out if isinstance(o, ItergpError)]
    if failed and errors == "raise":
        for o in out:
            if isinstance(o, Model):
                o.free()
        raise failed[0]
    return out


def autotune(n, d, p, kind="rbf", precision="bf16x3", items=False, lengthscale=1.0, stream=None):
    """Times every launch variant of the tensor-core product for this shape, records the
    fastest in the library's table; returns [(epilogue_warps, stages, cta_pair, ms)] and the
    best."""
    res = TuneResult()
    _check(lib.itergp_autotune(ct.byref(_kernel(kind, lengthscale, 1.0)), _prec(precision), int(n), int(d),
                               int(p), 1 if items else 0, ct.byref(res), _stream(stream)),
           "itergp_autotune")
    # (epilogue warps, stages (< 0: resident A), cta_pair, ms)
    vs = [(v.epilogue_warps, v.stages, v.cta_pair, v.ms) for v in res.variants[:res.count]]
    return vs, (vs[res.best] if res.best >= 0 else None)


def selftest_wait(limit_ns=20_000_000, stream=None):
    """Launch the bounded-wait self-test (a wait that runs out after limit_ns); the device
    status then reads ETIMEOUT (see sync_status)."""
    _check(lib.itergp_selftest_wait(int(limit_ns), _stream(stream)), "itergp_selftest_wait")


PROBES = {"ex2": 0, "ffma": 1, "mma_ss_n128": 2, "mma_ss_n256": 3, "mma_ss_n128_tmem_ld": 4,
          "mma_ts_n80": 5, "mma_ss_n128_tf32": 6, "dfma": 7, "rsqrt": 8,
          "pair_mma_ss_n128_f16": 9, "pair_mma_ss_n256_f16": 10, "pair_mma_ts_n80": 11,
          "pair_mma_ss_n192_f16": 12, "ring_pair_n128": 13, "ring_pair_n192": 14}
_PROBE_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libitergp_probe.so")
_probe_lib = None


def probe_lib():
    """The bench's throughput-probe library (libitergp_probe.so), loaded on first use."""
    global _probe_lib
    if _probe_lib is None:
        if not os.path.exists(_PROBE_LIB_PATH):
            raise ImportError(f"libitergp_probe.so not built ({_PROBE_LIB_PATH})")
        pl = ct.CDLL(_PROBE_LIB_PATH)
        pl.itergp_probe_throughput.argtypes = [ct.c_int32, ct.POINTER(ct.c_double), ct.c_void_p]
        pl.itergp_probe_throughput.restype = ct.c_int
        _probe_lib = pl
    return _probe_lib


def probe_throughput(what="ex2", stream=None) -> float:
    """Measured operations per second over the GPU (include/itergp_probe.h): MUFU exp2
    ("ex2"), FP32 FFMA ("ffma", flops), tcgen05.mma flops in the one-CTA product's shapes
    ("mma_ss_n128", "mma_ss_n256", "mma_ss_n128_tmem_ld": N = 128 while other warps stream
    TMEM loads, "mma_ts_n80", TF32 "mma_ss_n128_tf32") and in the CTA-pair form's
    ("pair_mma_ss_n128_f16", "pair_mma_ss_n256_f16", "pair_mma_ts_n80"), FP64 DFMA flops
    ("dfma") or MUFU rsqrt ("rsqrt")."""
    out = ct.c_double()
    _check(probe_lib().itergp_probe_throughput(PROBES[what], ct.byref(out), _stream(stream)),
           "itergp_probe_throughput")
    return out.value


def tune_save(path):
    """Write the launch-variant table as text lines (see include/itergp.h)."""
    _check(lib.itergp_tune_save(str(path).encode()), "itergp_tune_save")


def tune_load(path):
    """Merge a text table written by tune_save into the library's table."""
    _check(lib.itergp_tune_load(str(path).encode()), "itergp_tune_load")


def tune_clear():
    """Empty the launch-variant table (untuned launches use the defaults)."""
    _check(lib.itergp_tune_clear(), "itergp_tune_clear")


class Server:
    """Request loop over resident models (itergp_server_*): fits and predicts are queued
    from host arrays, run in batches on the GPU by the library's own threads, and report
    completion events.  Predict results land in NumPy arrays owned by this object until
    the request completes (``result(request_id)``)."""

    def __init__(self, model_bytes, work_bytes, precision="bf16x3", kind="rbf", d_max=32,
                 c_max=5, max_fit_batch=64, max_predict_batch=256, max_predict_rows=1 << 16,
                 max_newton=5, max_iters=5, rank=50, graph=True, tol_abs=1e-5, tol_rel=1e-5):
        import numpy as np
        self._np = np
        cfg = ServerConfig(int(model_bytes), int(work_bytes), KERNELS[kind], _prec(precision),
                           int(d_max), int(c_max), int(max_fit_batch), int(max_predict_batch),
                           int(max_predict_rows), int(max_newton), int(max_iters), int(rank),
                           1 if graph else 0, float(tol_abs), float(tol_rel))
        h = ct.c_void_p()
        _check(lib.itergp_server_create(ct.byref(cfg), ct.byref(h)), "itergp_server_create")
        self._h = h
        self._c = {}          # model id -> classes
        self._out = {}        # request id -> (mean, var, probs, inputs kept alive)

    def submit_fit(self, X, y, c, lengthscale=1.0, outputscale=1.0) -> int:
        """Queue a fit of host arrays X (n x d) and labels y; returns the model id.  The
        data are copied before the call returns."""
        np = self._np
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.int32)
        mid = ct.c_int64()
        _check(lib.itergp_server_submit_fit(self._h, X.ctypes.data, y.ctypes.data, X.shape[0],
                                            X.shape[1], int(c), float(lengthscale),
                                            float(outputscale), ct.byref(mid)),
               "itergp_server_submit_fit")
        self._c[mid.value] = int(c)
        return mid.value

    def submit_predict(self, model_id, Xs, var=True, probs=True) -> int:
        """Queue a predict against a model (it waits for the model's fit); returns the
        request id.  Its outputs land in host buffers read back with result()."""
        np = self._np
        Xs = np.ascontiguousarray(Xs, dtype=np.float32)
        c = self._c[model_id]
        mean = np.empty((Xs.shape[0], c), dtype=np.float32)
        v = np.empty_like(mean) if var else None
        p = np.empty_like(mean) if probs else None
        rid = ct.c_int64()
        _check(lib.itergp_server_submit_predict(self._h, int(model_id), Xs.ctypes.data, Xs.shape[0],
                                                mean.ctypes.data, v.ctypes.data if var else None,
                                                p.ctypes.data if probs else None, ct.byref(rid)),
               "itergp_server_submit_predict")
        self._out[rid.value] = (mean, v, p)
        return rid.value

    def poll(self, timeout_s=0.0, capacity=4096):
        """Completion events [(id, model, kind, status, submit_s, start_s, done_s, batch)]."""
        evs = (ServerEvent * capacity)()
        n = ct.c_int32()
        _check(lib.itergp_server_poll(self._h, evs, capacity, ct.byref(n),
                                      -1 if timeout_s is None else int(timeout_s * 1e6)),
               "itergp_server_poll")
        return [(e.id, e.model, e.kind, e.status, e.submit_s, e.start_s, e.done_s, e.batch)
                for e in evs[:n.value]]

    def result(self, request_id):
        """(mean, var, probs) of a completed predict (and forgets it)."""
        return self._out.pop(request_id)

    def release(self, model_id):
        """Drop a resident model once its queued predicts are done."""
        _check(lib.itergp_server_release(self._h, int(model_id)), "itergp_server_release")

    def stats(self) -> dict:
        """Resident models and rows, completed work and queue lengths."""
        st = ServerStats()
        _check(lib.itergp_server_get_stats(self._h, ct.byref(st)), "itergp_server_get_stats")
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def close(self):
        """Stop the request loop and free the server's device memory."""
        if self._h:
            _check(lib.itergp_server_destroy(self._h), "itergp_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
