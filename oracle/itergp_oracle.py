"""Plain FP64 CPU oracle for IterNCGP (Tatzel, Wenger, Schneider, Hennig:
"Accelerating Non-Conjugate Gaussian Processes By Trading Off Computation For
Uncertainty", arXiv 2310.20285).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import it; the product path (the C-ABI library and its
Python binding) never does, and it shares no code, header, table or helper with it.

Everything is float64 NumPy.  Library primitives (matmul, eigh, Cholesky) serve as single
steps; there is no blocking, fusion or reordering beyond what the paper's definitions and
algorithms state.  Vectors over the training set are stored as N x C arrays in the
paper's "CN ordering" (App. B.1): the class index moves fastest when flattened, so the
flattened vector is ``a.reshape(-1)``.

Readings of points where the paper is silent (each is listed in the design notes too):

* kernels (App. C.1/C.3 use GPyTorch RBF / Matern-3/2 with lengthscale l and
  outputscale s): RBF k = s exp(-r^2 / (2 l^2)); Matern-3/2 k = s (1 + sqrt3 r / l)
  exp(-sqrt3 r / l); r^2 = max(0, |a|^2 + |b|^2 - 2 a.b).
* W^-1 in Alg. 1-3 is read as the pseudo-inverse W^+ for the softmax likelihood
  (footnote to Eq. 6 and Lemma A.6).
* Alg. 3 "M = U Lambda U" is read as U Lambda U^T; M is used through its symmetric part;
  eigenpairs with lambda <= 1e-12 lambda_max are dropped before truncating to R.
* the inner stopping test is taken on r_{j-1} at the top of iteration j; eta_j <= 0
  stops the solver and the action s_j is not kept (App. B.2).
* unit-vector policy: action j of a Newton step is e_{B0 + j}, B0 = number of buffer
  columns left by the virtual solver run (so recycled unit actions are not repeated).
* exact Newton (the oracle's ground truth) solves the pseudo-target system with a
  Cholesky factor of  K_hat + gamma (I_N kron 11^T / C): the shift acts only on the
  per-point class-sum directions, which the right-hand side never touches.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RBF = 0
MATERN32 = 1


@dataclass(frozen=True)
class Kernel:
    """Stationary kernel with one lengthscale and outputscale, shared by all C outputs
    (independent GPs per class, App. C.3)."""
    kind: int = RBF
    lengthscale: float = 1.0
    outputscale: float = 1.0


@dataclass(frozen=True)
class ClassKernels:
    """One kernel per output: the C latent GPs are independent (Sec. 5, large-scale
    experiment; App. C.3) and each may carry its own hyperparameters (l_c, s_c).  The
    prior covariance is then K = sum_c k_c(X, X) kron e_c e_c^T in CN ordering, i.e. the
    block of class c acts on the class-c entries only."""
    kernels: tuple


def kernels_per_class(kern, C: int) -> list:
    """The kernel of each of the C outputs (the shared one C times)."""
    if isinstance(kern, ClassKernels):
        if len(kern.kernels) != C:
            raise ValueError("one kernel per class expected")
        return list(kern.kernels)
    return [kern] * C


# ---------------------------------------------------------------------------------------
# Kernel evaluation (Sec. 2.1 prior; App. C.1, C.3 kernels)
# ---------------------------------------------------------------------------------------

def sqdist(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Squared Euclidean distances r^2_ij = max(0, |a_i|^2 + |b_j|^2 - 2 a_i . b_j)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    na = np.einsum("ij,ij->i", A, A)
    nb = np.einsum("ij,ij->i", B, B)
    return np.maximum(na[:, None] + nb[None, :] - 2.0 * (A @ B.T), 0.0)


def kernel_of_sqdist(r2: np.ndarray, kern: Kernel) -> np.ndarray:
    """k as a function of r^2 (RBF, Matern-3/2)."""
    ell, s = float(kern.lengthscale), float(kern.outputscale)
    if kern.kind == RBF:
        return s * np.exp(-r2 / (2.0 * ell * ell))
    if kern.kind == MATERN32:
        u = math.sqrt(3.0) * np.sqrt(r2) / ell
        return s * (1.0 + u) * np.exp(-u)
    raise ValueError(f"unknown kernel kind {kern.kind}")


def kernel_matrix(A: np.ndarray, B: np.ndarray, kern: Kernel) -> np.ndarray:
    """k(A, B), dense M x N."""
    return kernel_of_sqdist(sqdist(A, B), kern)


def kmatvec(A: np.ndarray, B: np.ndarray, S: np.ndarray, kern: Kernel) -> np.ndarray:
    """Y = k(A, B) S for S of shape N x P (the lazily evaluated product of App. B.3.1;
    for the multi-output prior K = k kron I_C in CN ordering, K w = k(X, X) w with w
    viewed as N x C)."""
    return kernel_matrix(A, B, kern) @ np.asarray(S, dtype=np.float64)


def kmatvec_fp32(A: np.ndarray, B: np.ndarray, S: np.ndarray, kern: Kernel) -> np.ndarray:
    """The same product in FP32 arithmetic throughout (distances, kernel values and the
    weighted sum), K never stored beyond the block of rows of A passed in: the timed FP32
    baseline of the matrix-free product.  Not used as a reference."""
    A = np.asarray(A, dtype=np.float32)
    B = np.asarray(B, dtype=np.float32)
    na = np.einsum("ij,ij->i", A, A)
    nb = np.einsum("ij,ij->i", B, B)
    r2 = np.maximum(na[:, None] + nb[None, :] - np.float32(2.0) * (A @ B.T), np.float32(0.0))
    ell, s = np.float32(kern.lengthscale), np.float32(kern.outputscale)
    if kern.kind == RBF:
        k = s * np.exp(-r2 / (np.float32(2.0) * ell * ell))
    elif kern.kind == MATERN32:
        u = np.float32(math.sqrt(3.0)) * np.sqrt(r2) / ell
        k = s * (np.float32(1.0) + u) * np.exp(-u)
    else:
        raise ValueError(f"unknown kernel kind {kern.kind}")
    return k @ np.asarray(S, dtype=np.float32)


def dense_K(X: np.ndarray, C: int, kern) -> np.ndarray:
    """K = k(X, X) kron I_C in CN ordering (NC x NC), for tiny problems only; with one
    kernel per class, K = sum_c k_c(X, X) kron e_c e_c^T."""
    return cross_K(X, X, C, kern)


def cross_K(A: np.ndarray, B: np.ndarray, C: int, kern) -> np.ndarray:
    """The multi-output cross covariance between A and B in CN ordering ((M C) x (N C))."""
    out = 0.0
    for c, kc in enumerate(kernels_per_class(kern, C)):
        E = np.zeros((C, C))
        E[c, c] = 1.0
        out = out + np.kron(kernel_matrix(A, B, kc), E)
    return out


def kmatvec_classes(A: np.ndarray, B: np.ndarray, S: np.ndarray, kern, C: int) -> np.ndarray:
    """Y[:, j] = k_{j mod C}(A, B) S[:, j]: the product with the multi-output prior when the
    P columns of S are NC-vectors viewed as N x C blocks side by side (column j belongs to
    class j mod C, the CN ordering)."""
    S = np.asarray(S, dtype=np.float64)
    Y = np.zeros((np.asarray(A).shape[0], S.shape[1]))
    for c, kc in enumerate(kernels_per_class(kern, C)):
        Y[:, c::C] = kernel_matrix(A, B, kc) @ S[:, c::C]
    return Y


# ---------------------------------------------------------------------------------------
# Likelihoods: gradient and (pseudo-)inverse negative Hessian W
# ---------------------------------------------------------------------------------------

def softmax(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    e = np.exp(f - f.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def logsumexp(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    mx = f.max(axis=1)
    return mx + np.log(np.exp(f - mx[:, None]).sum(axis=1))


class Softmax:
    """Categorical likelihood with softmax inverse link (Sec. 2.1, App. A.6)."""

    def __init__(self, y: np.ndarray, C: int):
        self.y = np.asarray(y, dtype=np.int64)
        self.C = int(C)

    def onehot(self) -> np.ndarray:
        e = np.zeros((len(self.y), self.C))
        e[np.arange(len(self.y)), self.y] = 1.0
        return e

    def loglik(self, f):
        f = np.asarray(f, dtype=np.float64)
        return float(np.sum(f[np.arange(len(self.y)), self.y] - logsumexp(f)))

    def grad(self, f):
        """grad log p(y|f) = e_{y_n} - pi_n per data point (R&W Eq. 3.38 context)."""
        return self.onehot() - softmax(f)

    def W_blocks(self, f):
        """W_n = diag(pi_n) - pi_n pi_n^T, the CN-ordered diagonal blocks of W (Lemma A.6
        proof)."""
        pi = softmax(f)
        return np.einsum("nc,cd->ncd", pi, np.eye(self.C)) - np.einsum("nc,nd->ncd", pi, pi)

    def inv_pi(self, f):
        """1 / pi computed as exp(logsumexp(f) - f) (finite wherever pi underflows)."""
        f = np.asarray(f, dtype=np.float64)
        return np.exp(logsumexp(f)[:, None] - f)

    def Winv_apply(self, f, x):
        """W^+ x with W_n^+ = P diag(1/pi_n) P, P = I - 11^T / C (Lemma A.6); O(NC)."""
        x = np.asarray(x, dtype=np.float64)
        px = x - x.mean(axis=1, keepdims=True)
        q = px * self.inv_pi(f)
        return q - q.mean(axis=1, keepdims=True)

    def Winv_dense(self, f):
        N, C = len(self.y), self.C
        P = np.eye(C) - np.ones((C, C)) / C
        ip = self.inv_pi(f)
        out = np.zeros((N * C, N * C))
        for n in range(N):
            out[n * C:(n + 1) * C, n * C:(n + 1) * C] = P @ np.diag(ip[n]) @ P
        return out


class Gaussian:
    """Gaussian likelihood N(y; f, sigma^2 I) -- the conjugate special case of Thm. A.2:
    W^-1 = sigma^2 I and the pseudo targets equal y."""

    def __init__(self, y: np.ndarray, noise: float):
        self.y = np.asarray(y, dtype=np.float64)
        if self.y.ndim == 1:
            self.y = self.y[:, None]
        self.C = self.y.shape[1]
        self.noise = float(noise)

    def loglik(self, f):
        r = self.y - f
        return float(-0.5 * np.sum(r * r) / self.noise)

    def grad(self, f):
        return (self.y - f) / self.noise

    def Winv_apply(self, f, x):
        return self.noise * np.asarray(x, dtype=np.float64)

    def Winv_dense(self, f):
        return self.noise * np.eye(self.y.size)


class Bernoulli:
    """Binary classification with one latent function and the logistic inverse link
    pi = 1 / (1 + e^-f) (App. C, binary classification with one latent function):
    y in {0, 1}, log p(y|f) = sum_n y_n f_n - log(1 + e^f_n), grad = y - pi,
    W = diag(pi (1 - pi)), so W^-1 = diag(1 / (pi (1 - pi))) = diag(2 + e^f + e^-f)."""

    def __init__(self, y: np.ndarray):
        self.y = np.asarray(y, dtype=np.float64).reshape(-1, 1)
        self.C = 1

    def loglik(self, f):
        f = np.asarray(f, dtype=np.float64).reshape(-1, 1)
        return float(np.sum(self.y * f - np.logaddexp(0.0, f)))

    def grad(self, f):
        f = np.asarray(f, dtype=np.float64).reshape(-1, 1)
        return self.y - 1.0 / (1.0 + np.exp(-f))

    def winv_diag(self, f):
        f = np.asarray(f, dtype=np.float64).reshape(-1, 1)
        return 2.0 + np.exp(f) + np.exp(-f)

    def Winv_apply(self, f, x):
        return self.winv_diag(f) * np.asarray(x, dtype=np.float64).reshape(-1, 1)

    def Winv_dense(self, f):
        return np.diag(self.winv_diag(f).reshape(-1))


class Poisson:
    """Count regression with the log link (App. A, derivatives of the Poisson log
    likelihood): rate lambda = e^f, log p(y|f) = sum_n y_n f_n - e^f_n (the constant
    -log y_n! is dropped), grad = y - e^f, W = diag(e^f), W^-1 = diag(e^-f)."""

    def __init__(self, y: np.ndarray):
        self.y = np.asarray(y, dtype=np.float64).reshape(-1, 1)
        self.C = 1

    def loglik(self, f):
        f = np.asarray(f, dtype=np.float64).reshape(-1, 1)
        return float(np.sum(self.y * f - np.exp(f)))

    def grad(self, f):
        return self.y - np.exp(np.asarray(f, dtype=np.float64).reshape(-1, 1))

    def winv_diag(self, f):
        return np.exp(-np.asarray(f, dtype=np.float64).reshape(-1, 1))

    def Winv_apply(self, f, x):
        return self.winv_diag(f) * np.asarray(x, dtype=np.float64).reshape(-1, 1)

    def Winv_dense(self, f):
        return np.diag(self.winv_diag(f).reshape(-1))


# ---------------------------------------------------------------------------------------
# Exact Newton (the plain definition, Eqs. 3 and 6-7 / Prop. A.1)
# ---------------------------------------------------------------------------------------

def pseudo_targets(lik, f):
    """y_hat = f + W^-1 grad log p(y | f)  (Alg. 1 / Eq. 6)."""
    return np.asarray(f, dtype=np.float64) + lik.Winv_apply(f, lik.grad(f))


def exact_newton_step(X, lik, f, m, kern: Kernel, shift: float | None = None):
    """One exact Newton step through the pseudo-target system (Eqs. 6-7):
    v = (K + W^+)^-1 (y_hat - m),  f_next = K v + m.

    The system is solved with a Cholesky factor of K_hat + gamma (I_N kron 11^T / C);
    gamma defaults to the outputscale.  For the softmax likelihood the right-hand side
    has zero class-sum per data point, W^+ vanishes on the class-sum directions and
    K = k kron I_C maps them to themselves, so the shift leaves v unchanged while making
    the factorisation well conditioned.  For C = 1 / other likelihoods use shift=0."""
    N, C = f.shape
    K = dense_K(X, C, kern)
    Khat = K + lik.Winv_dense(f)
    # with one kernel per class K no longer maps the class-sum directions to themselves,
    # so no shift is applied (K + W^+ is positive definite when every k_c is)
    gamma = (0.0 if isinstance(kern, ClassKernels) else kern.outputscale) if shift is None else shift
    if gamma:
        Khat = Khat + gamma * np.kron(np.eye(N), np.ones((C, C)) / C)
    b = (pseudo_targets(lik, f) - m).reshape(-1)
    L = np.linalg.cholesky(Khat)
    v = np.linalg.solve(L.T, np.linalg.solve(L, b))
    f_next = (K @ v).reshape(N, C) + m
    return v.reshape(N, C), f_next


def exact_newton(X, lik, C, kern: Kernel, steps: int, shift: float | None = None):
    N = len(X)
    m = np.zeros((N, C))
    f = m.copy()
    fs, vs = [f], []
    for _ in range(steps):
        v, f = exact_newton_step(X, lik, f, m, kern, shift)
        fs.append(f)
        vs.append(v)
    return fs, vs


def contrast_condition(X, lik, f, kern: Kernel, C: int) -> float:
    """Condition number of K_hat = K + W^+ restricted to the class contrasts range(I kron P),
    the subspace the softmax solves live in (reading of Lemma A.6: W^+ vanishes on the
    per-point class sums).  Dense FP64 eigenvalues of B^T K_hat B, with B an orthonormal
    basis of range(I kron P); for tiny N only.  It bounds how far FP32 products can move a
    solve on this subspace."""
    N = len(X)
    Khat = dense_K(X, C, kern) + lik.Winv_dense(f)
    P = np.eye(C) - np.ones((C, C)) / C
    w, V = np.linalg.eigh(P)
    Bc = V[:, w > 0.5]                       # the C - 1 unit eigenvectors of the projector
    B = np.kron(np.eye(N), Bc)
    lam = np.linalg.eigvalsh(B.T @ Khat @ B)
    return float(lam.max() / lam.min())


def objective(lik, f, v, m):
    """Psi(f) = log p(y|f) - 1/2 (f - m)^T K^-1 (f - m)  (Eq. 2), evaluated without K^-1
    through f - m = K v (Prop. A.1): (f - m)^T K^-1 (f - m) = v^T (f - m)."""
    return lik.loglik(f) - 0.5 * float(np.sum(np.asarray(v) * (np.asarray(f) - m)))


# ---------------------------------------------------------------------------------------
# IterGP inner loop (Alg. 2) with the virtual solver run and compression (Alg. 3)
# ---------------------------------------------------------------------------------------

CG = 0
UNIT = 1

STOP_MAXITER = 0
STOP_TOL = 1
STOP_ETA = 2


def virtual_solver_run(S, T, winv_cols, R: int | None, drop_rel: float = 1e-12):
    """Alg. 3.  S, T: NC x B (T = K S).  Returns (Q0, S, T, n_dropped).

    M = S^T (T + W^-1 S); eigendecomposition M = U Lambda U^T with lambda descending;
    optional truncation to the R largest eigenpairs; S <- S U, T <- T U;
    Q0 = S Lambda^-1/2 (root of C0 = Q0 Q0^T)."""
    B = S.shape[1]
    if B == 0:
        return np.zeros_like(S), S, T, 0
    M = S.T @ (T + winv_cols(S))
    M = 0.5 * (M + M.T)
    lam, U = np.linalg.eigh(M)
    order = np.argsort(-lam, kind="stable")
    lam, U = lam[order], U[:, order]
    keep = lam > drop_rel * max(lam[0], 0.0)
    n_dropped = int(np.count_nonzero(~keep))
    lam, U = lam[keep], U[:, keep]
    if R is not None:
        lam, U = lam[:R], U[:, :R]
    S = S @ U
    T = T @ U
    Q0 = S / np.sqrt(lam)[None, :]
    return Q0, S, T, n_dropped


@dataclass
class SolveInfo:
    iters: int = 0
    stop: int = STOP_MAXITER
    rnorm: list = field(default_factory=list)
    B0: int = 0
    dropped: int = 0


def itergp(kmv, winv, b, S, T, policy: int = CG, max_iters: int = 50,
           R: int | None = None, tol_abs: float = 1e-5, tol_rel: float = 1e-5,
           on_iterate=None, project=None):
    """Alg. 2: IterGP with a virtual solver run.

    kmv(w)  -- product with K for an NC-vector (flat, CN order)
    winv(w) -- product with W^-1 (W^+ for softmax) for an NC-vector (flat)
    b       -- right-hand side y_hat - m (flat)
    S, T    -- action buffer and its K products (NC x B), recycled from earlier steps.
    Returns (v, Q, S, T, info); C_j = Q Q^T.  ``on_iterate(j, v, Q)`` is called after
    every completed iteration (used by tests of the per-iteration invariants).
    ``project`` (optional) is applied to each residual; the CUDA path projects onto the
    class-contrast subspace, which is the identity on residuals in exact arithmetic."""
    NC = b.shape[0]

    def winv_cols(Mat):
        return np.stack([winv(Mat[:, k]) for k in range(Mat.shape[1])], axis=1) \
            if Mat.shape[1] else Mat

    Q, S, T, dropped = virtual_solver_run(S, T, winv_cols, R)
    v = Q @ (Q.T @ b)                                        # v0 = C0 (y_hat - m)
    info = SolveInfo(B0=S.shape[1], dropped=dropped)
    bnorm = float(np.linalg.norm(b))
    thresh = max(tol_abs, tol_rel * bnorm)
    for j in range(1, max_iters + 1):
        r = b - kmv(v) - winv(v)                            # r_{j-1}
        if project is not None:
            r = project(r)
        rn = float(np.linalg.norm(r))
        info.rnorm.append(rn)
        if rn < thresh:
            info.stop = STOP_TOL
            break
        if policy == CG:
            s = r.copy()                                    # residual action (CG)
        else:
            s = np.zeros(NC)
            idx = info.B0 + j - 1                           # e_{B0 + j}
            if idx >= NC:
                info.stop = STOP_MAXITER
                break
            s[idx] = 1.0
        alpha = float(s @ r)                                # observation alpha_j
        t = kmv(s)                                          # t_j = K s_j
        z = t + winv(s)                                     # z_j = K_hat s_j
        d = s - Q @ (Q.T @ z)                               # d_j = s_j - C_{j-1} z_j
        eta = float(z @ d)                                  # eta_j = z_j^T d_j
        if eta <= 0.0:
            info.stop = STOP_ETA
            break
        S = np.concatenate([S, s[:, None]], axis=1)
        T = np.concatenate([T, t[:, None]], axis=1)
        Q = np.concatenate([Q, (d / math.sqrt(eta))[:, None]], axis=1)
        v = v + (alpha / eta) * d
        info.iters = j
        if on_iterate is not None:
            on_iterate(j, v, Q)
    return v, Q, S, T, info


# ---------------------------------------------------------------------------------------
# IterNCGP outer loop (Alg. 1)
# ---------------------------------------------------------------------------------------

@dataclass
class FitResult:
    v: np.ndarray            # representer weights, N x C
    Q: np.ndarray            # root of C_j, NC x B
    f: np.ndarray            # latest Newton iterate f_{i+1}, N x C
    fs: list                 # f_0, f_1, ...
    objectives: list         # Psi(f_i) per step
    rel_changes: list        # |g_i - g_{i-1}| / |g_i| per step (i >= 1)
    infos: list              # SolveInfo per Newton step
    newton_steps: int = 0


def iterncgp_fit(X, lik, C: int, kern: Kernel, max_newton: int = 10, max_iters: int = 50,
                 R: int | None = None, policy: int = CG, tol_newton: float | None = None,
                 tol_abs: float = 1e-5, tol_rel: float = 1e-5, recycle: bool = True,
                 project_contrasts: bool = False, f0=None, product_noise=None):
    """Alg. 1: Newton's method as a sequence of GP regression problems, each solved by
    IterGP (Alg. 2) with recycled actions (Alg. 3).  Prior mean m = 0 (App. C.3),
    f_0 = m, empty buffers.  tol_newton=None runs exactly ``max_newton`` steps.
    project_contrasts=True removes the per-point class mean from y_hat - m and from every
    residual under the residual (CG) policy (the CUDA path's stabilisation; the identity
    in exact arithmetic, where those vectors already lie in range(I kron P)).
    f0 (N x C) replaces the starting iterate f_0 = m (used to start a step from a given
    iterate); the objective of step 0 is then reported with v = 0 as for f_0 = m.
    product_noise=(eps, rng) models an inexact kernel product: every application of K
    (each solver product and f = K v) returns (K W)(1 + eps z) with z standard normal,
    drawn fresh from rng per call, as rounding of relative size eps would.  Off (None) by
    default; tests use it to measure how far rounding of a given size moves a fit."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    m = np.zeros((N, C))
    f = m.copy() if f0 is None else np.array(f0, dtype=np.float64).reshape(N, C)
    S = np.zeros((N * C, 0))
    T = np.zeros((N * C, 0))
    v = np.zeros((N, C))
    Q = np.zeros((N * C, 0))
    res = FitResult(v, Q, f, [f.copy()], [], [], [])
    per_class = isinstance(kern, ClassKernels)
    kx = None if per_class else kernel_matrix(X, X, kern)
    kxs = [kernel_matrix(X, X, kc) for kc in kernels_per_class(kern, C)] if per_class else None

    def kprod_exact(W):   # K applied to an N x C block (k kron I_C, or class c's kernel on column c)
        if not per_class:
            return kx @ W
        return np.stack([kxs[c] @ W[:, c] for c in range(C)], axis=1)

    def kprod(W):
        Y = kprod_exact(W)
        if product_noise is None:
            return Y
        eps, rng = product_noise
        return Y * (1.0 + eps * rng.standard_normal(Y.shape))

    def kmv(w):
        return kprod(w.reshape(N, C)).reshape(-1)

    g_prev = None
    v_prev = np.zeros((N, C))
    for i in range(max_newton):
        g = f - m
        res.objectives.append(objective(lik, f, v_prev, m))
        if g_prev is not None:
            gn = float(np.linalg.norm(g))
            rc = float(np.linalg.norm(g - g_prev)) / gn if gn > 0 else 0.0
            res.rel_changes.append(rc)
            if tol_newton is not None and rc <= tol_newton:
                break
        winv = (lambda w, f=f: lik.Winv_apply(f, w.reshape(N, C)).reshape(-1))
        yhat = pseudo_targets(lik, f)
        b = (yhat - m).reshape(-1)
        proj = None
        if project_contrasts and policy == CG:
            proj = (lambda w: (w.reshape(N, C) - w.reshape(N, C).mean(axis=1, keepdims=True)).reshape(-1))
            b = proj(b)
        if not recycle:
            S = np.zeros((N * C, 0))
            T = np.zeros((N * C, 0))
        vflat, Q, S, T, info = itergp(kmv, winv, b, S, T, policy, max_iters, R,
                                      tol_abs, tol_rel, project=proj)
        v = vflat.reshape(N, C)
        f = kprod(v) + m                                    # f_{i+1} = K v + m
        res.fs.append(f.copy())
        res.infos.append(info)
        res.newton_steps = i + 1
        g_prev = g
        v_prev = v
    res.v, res.Q, res.f = v, Q, f
    return res


# ---------------------------------------------------------------------------------------
# Posterior predictive (Eqs. 9-10) and probit approximation (App. C.3)
# ---------------------------------------------------------------------------------------

def predict(Xs, X, v, Q, kern, C: int):
    """mean m(x*) + k(x*, X) v (m = 0); marginal variance
    diag k_{i,j}(x*, x*) = s - sum_b ((k(x*, X) Q_b)_c)^2 (Eq. 10 with C_j = Q Q^T, as in
    the proof of Prop. A.3); probit probabilities softmax(mean / sqrt(1 + pi/8 var)).
    With one kernel per class, column c uses k_c and s_c."""
    N = X.shape[0]
    ks = kernels_per_class(kern, C)
    kx = [kernel_matrix(Xs, X, kc) for kc in ks]
    v = np.asarray(v, dtype=np.float64)
    mean = np.stack([kx[c] @ v[:, c] for c in range(C)], axis=1)
    var = np.tile(np.array([float(kc.outputscale) for kc in ks]), (mean.shape[0], 1))
    for b in range(Q.shape[1]):
        Qb = Q[:, b].reshape(N, C)
        proj = np.stack([kx[c] @ Qb[:, c] for c in range(C)], axis=1)
        var -= proj * proj
    probs = softmax(mean / np.sqrt(1.0 + (math.pi / 8.0) * var))
    return mean, var, probs


def exact_predict(Xs, X, lik, f_i, f_next, kern: Kernel, C: int,
                  contrasts_only: bool = True):
    """The exact Laplace predictive (Eqs. 4-5) at Newton iterate f_i, dense, tiny N.

    mean = k(x*, X) K^-1 (f_{i+1} - m)  (Eq. 4, m = 0)
    cov  = k(x*, x*) - k(x*, X) K_hat^-1 k(X, x*),  K_hat = K + W^+  (Eq. 5)

    With the softmax pseudo-inverse, W^+ is zero on the per-point class-sum directions,
    so the literal Eq. 5 conditions those directions as if they were observed without
    noise.  ``contrasts_only=False`` returns that literal form (what IterGP reaches with
    all NC unit-vector actions); ``contrasts_only=True`` restricts K_hat^-1 to the
    class-contrast subspace range(I_N kron P), which is the limit of residual (CG)
    actions and equals the Laplace predictive k - k (K^-1 + W)^-1-form with W singular.
    Returns the mean and the marginal variances (M x C)."""
    N = X.shape[0]
    K = dense_K(X, C, kern)
    Kx = cross_K(Xs, X, C, kern)                             # (M C) x (N C)
    mean = Kx @ np.linalg.solve(K, np.asarray(f_next, dtype=np.float64).reshape(-1))
    Khat = K + lik.Winv_dense(f_i)
    ks = kernels_per_class(kern, C)
    if contrasts_only:
        Pi = np.kron(np.eye(N), np.eye(C) - np.ones((C, C)) / C)
        Khat = Khat + ks[0].outputscale * np.kron(np.eye(N), np.ones((C, C)) / C)
        red = Kx @ Pi @ np.linalg.solve(Khat, Pi @ Kx.T)
    else:
        red = Kx @ np.linalg.solve(Khat, Kx.T)
    prior = np.tile(np.array([float(kc.outputscale) for kc in ks]), Xs.shape[0])
    var = prior - np.diag(red)
    return mean.reshape(-1, C), var.reshape(-1, C)
