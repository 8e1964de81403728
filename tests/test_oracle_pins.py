"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something that is not the oracle: a SciPy / NumPy
library routine computing the same definition another way, a closed form at special
points, textbook conjugate gradients, a dense formula from a different equation of the
paper, or an invariant the paper proves.  A plausible slip in the oracle (a dropped
term, a wrong sign, a transposed operand, a wrong lengthscale convention) fails at least
one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.spatial.distance
import scipy.special
import scipy.stats

import oracle.itergp_oracle as O
from paper_2310_20285_gb300 import datagen

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def tiny_problem(n=12, d=2, c=3, seed=7, ell=0.7, s=1.3, kind=O.RBF):
    X, y, _ = datagen.blobs(n, d, c, seed)
    return X, y, O.Kernel(kind, ell, s)


# ---------------------------------------------------------------------- kernel (L0)

def test_sqdist_matches_scipy_cdist():
    g = np.random.default_rng(0)
    A, B = g.standard_normal((17, 5)) * 3, g.standard_normal((9, 5))
    ref = scipy.spatial.distance.cdist(A, B, "sqeuclidean")
    assert np.allclose(O.sqdist(A, B), ref, rtol=1e-12, atol=1e-12)
    assert np.all(O.sqdist(A, A) >= 0.0)



def test_fp32_product_matches_the_brute_force_double_loop():
    """The FP32 timed baseline against a brute-force double loop in FP64, for both kernels:
    within FP32 rounding (1e-5 normwise)."""
    g = np.random.default_rng(3)
    A, B = g.standard_normal((23, 4)), g.standard_normal((31, 4))
    S = g.standard_normal((31, 5))
    for kern in (O.Kernel(O.RBF, 0.9, 1.3), O.Kernel(O.MATERN32, 1.7, 0.6)):
        ref = np.zeros((23, 5))
        for i in range(23):
            for j in range(31):
                r = float(np.sqrt(((A[i] - B[j]) ** 2).sum()))
                if kern.kind == O.RBF:
                    k = kern.outputscale * math.exp(-r * r / (2 * kern.lengthscale ** 2))
                else:
                    u = math.sqrt(3.0) * r / kern.lengthscale
                    k = kern.outputscale * (1 + u) * math.exp(-u)
                ref[i] += k * S[j]
        got = O.kmatvec_fp32(A, B, S, kern)
        assert got.dtype == np.float32
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)

def test_rbf_closed_form_points_and_gaussian_pdf():
    ell, s = 1.7, 2.5
    kern = O.Kernel(O.RBF, ell, s)
    r = np.array([0.0, ell, 2 * ell, 0.3])
    k = O.kernel_of_sqdist(r * r, kern)
    assert k[0] == pytest.approx(s)
    assert k[1] == pytest.approx(s * math.exp(-0.5))
    assert k[2] == pytest.approx(s * math.exp(-2.0))
    # k(r) = s * sqrt(2 pi) l * N(r; 0, l^2)
    ref = s * math.sqrt(2 * math.pi) * ell * scipy.stats.norm.pdf(r, scale=ell)
    assert np.allclose(k, ref, rtol=1e-13)


def test_matern32_against_general_matern_bessel_form():
    """Matern-nu kernel s 2^(1-nu)/Gamma(nu) (sqrt(2 nu) r/l)^nu K_nu(sqrt(2 nu) r/l) at
    nu = 3/2 (R&W Eq. 4.14) evaluated with scipy's modified Bessel function."""
    ell, s, nu = 0.8, 0.45, 1.5
    kern = O.Kernel(O.MATERN32, ell, s)
    r = np.linspace(0.05, 4.0, 37)
    u = math.sqrt(2 * nu) * r / ell
    ref = s * 2 ** (1 - nu) / scipy.special.gamma(nu) * u ** nu * scipy.special.kv(nu, u)
    assert np.allclose(O.kernel_of_sqdist(r * r, kern), ref, rtol=1e-12)
    assert O.kernel_of_sqdist(np.array([0.0]), kern)[0] == pytest.approx(s)
    # r = l: s (1 + sqrt3) e^-sqrt3
    assert O.kernel_of_sqdist(np.array([ell * ell]), kern)[0] == pytest.approx(
        s * (1 + math.sqrt(3)) * math.exp(-math.sqrt(3)))


@pytest.mark.parametrize("kind", [O.RBF, O.MATERN32])
def test_kernel_matrix_symmetric_psd_unit_diagonal(kind):
    X, _, kern = tiny_problem(n=40, d=3, kind=kind)
    K = O.kernel_matrix(X, X, kern)
    assert np.allclose(K, K.T, atol=0)
    assert np.allclose(np.diag(K), kern.outputscale, rtol=1e-12)
    assert np.linalg.eigvalsh(K).min() >= -1e-12 * kern.outputscale


@pytest.mark.parametrize("kind", [O.RBF, O.MATERN32])
def test_kmatvec_brute_force_double_loop(kind):
    g = np.random.default_rng(3)
    A, B = g.standard_normal((7, 4)), g.standard_normal((11, 4))
    S = g.standard_normal((11, 5))
    kern = O.Kernel(kind, 1.1, 0.9)
    Y = np.zeros((7, 5))
    for i in range(7):
        for j in range(11):
            r = math.sqrt(sum((A[i, d] - B[j, d]) ** 2 for d in range(4)))
            if kind == O.RBF:
                k = 0.9 * math.exp(-r * r / (2 * 1.1 ** 2))
            else:
                k = 0.9 * (1 + math.sqrt(3) * r / 1.1) * math.exp(-math.sqrt(3) * r / 1.1)
            Y[i] += k * S[j]
    assert np.allclose(O.kmatvec(A, B, S, kern), Y, rtol=1e-12, atol=1e-12)


def test_dense_K_is_block_diagonal_in_nc_ordering():
    X, _, kern = tiny_problem(n=5)
    C = 3
    K = O.dense_K(X, C, kern)
    k = O.kernel_matrix(X, X, kern)
    # CN ordering: entry (n*C + c, m*C + e) = k(x_n, x_m) delta_ce   (App. B.1)
    for n in range(5):
        for m in range(5):
            assert np.allclose(K[n * C:(n + 1) * C, m * C:(m + 1) * C], k[n, m] * np.eye(C))


# ---------------------------------------------------------------------- likelihood, W

def test_softmax_grad_matches_finite_differences_of_loglik():
    g = np.random.default_rng(5)
    N, C = 6, 4
    f = g.standard_normal((N, C))
    y = g.integers(0, C, N)
    lik = O.Softmax(y, C)
    h = 1e-6
    fd = np.zeros_like(f)
    for n in range(N):
        for c in range(C):
            e = np.zeros_like(f)
            e[n, c] = h
            fd[n, c] = (lik.loglik(f + e) - lik.loglik(f - e)) / (2 * h)
    assert np.allclose(lik.grad(f), fd, atol=1e-8)
    assert np.allclose(lik.grad(f).sum(axis=1), 0.0, atol=1e-14)


def test_W_blocks_equal_minus_hessian_by_finite_differences():
    g = np.random.default_rng(6)
    N, C = 3, 4
    f = g.standard_normal((N, C))
    lik = O.Softmax(g.integers(0, C, N), C)
    h = 1e-6
    W = lik.W_blocks(f)
    for n in range(N):
        for c in range(C):
            e = np.zeros_like(f)
            e[n, c] = h
            col = -(lik.grad(f + e) - lik.grad(f - e))[n] / (2 * h)
            assert np.allclose(W[n, :, c], col, atol=1e-8)
    assert np.allclose(W.sum(axis=2), 0.0, atol=1e-15)        # W_n 1 = 0


def test_W_pinv_closed_form_is_moore_penrose():
    """Lemma A.6: P diag(1/pi) P satisfies the four Moore-Penrose conditions and
    matches numpy's SVD pseudo-inverse; W W^+ = P."""
    g = np.random.default_rng(8)
    N, C = 5, 4
    f = 2 * g.standard_normal((N, C))
    lik = O.Softmax(g.integers(0, C, N), C)
    Wb = lik.W_blocks(f)
    P = np.eye(C) - np.ones((C, C)) / C
    Wd = lik.Winv_dense(f)
    for n in range(N):
        A = Wb[n]
        Ap = Wd[n * C:(n + 1) * C, n * C:(n + 1) * C]
        assert np.allclose(A @ Ap @ A, A, atol=1e-12)
        assert np.allclose(Ap @ A @ Ap, Ap, atol=1e-9 * np.abs(Ap).max())
        assert np.allclose((A @ Ap).T, A @ Ap, atol=1e-12)
        assert np.allclose((Ap @ A).T, Ap @ A, atol=1e-12)
        assert np.allclose(A @ Ap, P, atol=1e-12)
        assert np.allclose(Ap, np.linalg.pinv(A, rcond=1e-13), rtol=1e-8, atol=1e-9)
    x = g.standard_normal((N, C))
    assert np.allclose(lik.Winv_apply(f, x).reshape(-1), Wd @ x.reshape(-1), atol=1e-12)
    assert np.allclose(lik.Winv_apply(f, np.ones((N, C))), 0.0, atol=1e-12)


def test_inv_pi_is_reciprocal_softmax_for_tiny_probabilities():
    lik = O.Softmax(np.array([0]), 3)
    f = np.array([[300.0, 0.0, -10.0]])
    ip = lik.inv_pi(f)
    assert np.all(np.isfinite(ip))
    assert ip[0, 0] == pytest.approx(1.0)
    assert math.log(ip[0, 1]) == pytest.approx(300.0)
    assert math.log(ip[0, 2]) == pytest.approx(310.0)
    g = np.random.default_rng(0).standard_normal((4, 3))
    assert np.allclose(O.Softmax(np.zeros(4, int), 3).inv_pi(g), 1.0 / O.softmax(g))


# ---------------------------------------------------------------------- exact Newton

def textbook_newton_step(K, lik, f, m):
    """Eq. 3: f + (W + K^-1)^-1 (grad log p - K^-1 (f - m)), dense, W from its blocks."""
    N, C = f.shape
    W = scipy.linalg.block_diag(*lik.W_blocks(f))
    Kinv = np.linalg.inv(K)
    g = lik.grad(f).reshape(-1) - Kinv @ (f - m).reshape(-1)
    return f + np.linalg.solve(W + Kinv, g).reshape(N, C)


@pytest.mark.parametrize("kind", [O.RBF, O.MATERN32])
def test_exact_newton_pseudo_targets_equal_textbook_newton(kind):
    X, y, kern = tiny_problem(n=10, kind=kind, ell=0.6)
    C = 3
    lik = O.Softmax(y, C)
    K = O.dense_K(X, C, kern)
    m = np.zeros((10, C))
    f = m.copy()
    for _ in range(4):
        _, f_next = O.exact_newton_step(X, lik, f, m, kern)
        ref = textbook_newton_step(K, lik, f, m)
        assert np.allclose(f_next, ref, rtol=1e-8, atol=1e-9)
        f = f_next


def test_exact_newton_shift_does_not_change_solution():
    X, y, kern = tiny_problem(n=9, ell=0.5)
    lik = O.Softmax(y, 3)
    m = np.zeros((9, 3))
    f = np.random.default_rng(1).standard_normal((9, 3))
    f -= f.mean(axis=1, keepdims=True)
    v1, _ = O.exact_newton_step(X, lik, f, m, kern, shift=0.3)
    v2, _ = O.exact_newton_step(X, lik, f, m, kern, shift=5.0)
    assert np.allclose(v1, v2, atol=1e-9)


def test_exact_newton_shift_matches_lu_of_the_unshifted_system():
    """The shifted Cholesky reading of the exact step against the plain definition: an LU
    solve of the unshifted K_hat = K + W^+ (invertible at tiny N when k(X, X) is well
    conditioned, which a short lengthscale gives)."""
    import scipy.linalg as sla
    X, y, kern = tiny_problem(n=9, ell=0.3)
    lik = O.Softmax(y, 3)
    m = np.zeros((9, 3))
    f = np.random.default_rng(2).standard_normal((9, 3))
    f -= f.mean(axis=1, keepdims=True)        # Newton iterates f = K v have zero class sums
    K = O.dense_K(X, 3, kern)
    Khat = K + lik.Winv_dense(f)
    assert np.linalg.cond(Khat) < 1e6
    b = (O.pseudo_targets(lik, f) - m).reshape(-1)
    v_lu = sla.lu_solve(sla.lu_factor(Khat), b)
    v, f_next = O.exact_newton_step(X, lik, f, m, kern)          # default shift gamma = s
    assert np.allclose(v.reshape(-1), v_lu, rtol=1e-9, atol=1e-10)
    assert np.allclose(f_next.reshape(-1), K @ v_lu, rtol=1e-9, atol=1e-10)


def test_newton_converges_to_stationary_point():
    """At the mode grad Psi = 0, i.e. grad log p(y|f) = K^-1 (f - m) = v (Eq. 3, Prop. A.1)."""
    X, y, kern = tiny_problem(n=15, ell=1.0)
    lik = O.Softmax(y, 3)
    fs, vs = O.exact_newton(X, lik, 3, kern, steps=12)
    assert np.allclose(lik.grad(fs[-1]), vs[-1], atol=1e-9)
    # the objective (Eq. 2, evaluated through v) increases monotonically
    m = np.zeros_like(fs[0])
    K = O.dense_K(X, 3, kern)
    psi = [lik.loglik(f) - 0.5 * (f - m).reshape(-1) @ np.linalg.solve(K, (f - m).reshape(-1))
           for f in fs[1:]]
    psi_v = [O.objective(lik, f, v, m) for f, v in zip(fs[1:], vs)]
    assert np.allclose(psi, psi_v, rtol=1e-7)
    assert all(b >= a - 1e-9 for a, b in zip(psi, psi[1:]))


def test_objective_gradient_by_finite_differences_vanishes_at_the_newton_limit():
    """Brute force, independent of the identity grad log p = v: central differences of
    Psi(f) = log p(y|f) - 1/2 f^T K^-1 f (Eq. 2, m = 0, K^-1 by a dense solve) vanish at
    the exact Newton iteration's limit and not at its starting point."""
    X, y, kern = tiny_problem(n=6, ell=1.0)
    C = 3
    lik = O.Softmax(y, C)
    fs, _ = O.exact_newton(X, lik, C, kern, steps=15)
    K = O.dense_K(X, C, kern)

    def psi(fflat):
        return lik.loglik(fflat.reshape(-1, C)) - 0.5 * fflat @ np.linalg.solve(K, fflat)

    def fd_grad(f, h=1e-5):
        f = f.reshape(-1)
        g = np.zeros_like(f)
        for i in range(f.size):
            e = np.zeros_like(f)
            e[i] = h
            g[i] = (psi(f + e) - psi(f - e)) / (2 * h)
        return g

    assert np.max(np.abs(fd_grad(fs[-1]))) < 1e-6
    # after one step the gradient is still far from zero
    assert np.max(np.abs(fd_grad(fs[1]))) > 1e-3


def test_contrast_condition_lies_within_its_weyl_bounds():
    """On range(I kron P) the eigenvalues of K_hat lie in [min 1/pi, lambda_max(k) +
    max 1/pi] (W^+ = P diag(1/pi) P has Rayleigh quotients in [min 1/pi, max 1/pi] there
    and K = k kron I_C adds [0, lambda_max(k)]), so 1 <= cond <= (lambda_max(k) +
    max 1/pi) / min 1/pi along the whole Newton path; without K the condition is that of
    diag(1/pi) on the contrasts."""
    X, y, kern = tiny_problem(n=7, ell=0.9)
    C = 3
    lik = O.Softmax(y, C)
    fs, _ = O.exact_newton(X, lik, C, kern, steps=6)
    lam_k = float(np.linalg.eigvalsh(O.kernel_matrix(X, X, kern)).max())
    for f in fs:
        ip = lik.inv_pi(f)
        kappa = O.contrast_condition(X, lik, f, kern, C)
        assert 1.0 <= kappa <= (lam_k + ip.max()) / ip.min() * (1 + 1e-12)
    # K -> 0 (tiny outputscale): the bound tightens to the spread of 1/pi on the contrasts
    tiny = O.Kernel(kern.kind, kern.lengthscale, 1e-12)
    f = fs[-1]
    ip = lik.inv_pi(f)
    assert O.contrast_condition(X, lik, f, tiny, C) <= ip.max() / ip.min() * (1 + 1e-9)


# ---------------------------------------------------------------------- IterGP (Alg. 2)

def _system(n=10, c=3, seed=7, ell=0.6):
    X, y, kern = tiny_problem(n=n, c=c, seed=seed, ell=ell)
    lik = O.Softmax(y, c)
    f = np.random.default_rng(seed).standard_normal((n, c))
    f -= f.mean(axis=1, keepdims=True)
    K = O.dense_K(X, c, kern)
    Khat = K + lik.Winv_dense(f)
    b = (O.pseudo_targets(lik, f)).reshape(-1)
    kmv = lambda w: K @ w
    winv = lambda w: lik.Winv_apply(f, w.reshape(n, c)).reshape(-1)
    return K, Khat, b, kmv, winv


def test_unit_vector_actions_reproduce_the_direct_solve():
    """NC unit-vector actions span R^NC, so C_NC = K_hat^-1 (Eq. 11, Sec. 3.2)."""
    K, Khat, b, kmv, winv = _system()
    NC = b.size
    v, Q, S, T, info = O.itergp(kmv, winv, b, np.zeros((NC, 0)), np.zeros((NC, 0)),
                                policy=O.UNIT, max_iters=NC, tol_abs=0, tol_rel=0)
    assert info.iters == NC
    assert np.allclose(v, np.linalg.solve(Khat, b), rtol=1e-9, atol=1e-10)
    assert np.allclose(Q @ Q.T, np.linalg.inv(Khat), rtol=1e-7, atol=1e-9)


def textbook_cg(A, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    out = []
    for _ in range(iters):
        Ap = A @ p
        a = (r @ r) / (p @ Ap)
        x = x + a * p
        rn = r - a * Ap
        p = rn + (rn @ rn) / (r @ r) * p
        r = rn
        out.append(x.copy())
    return out


def test_residual_actions_equal_conjugate_gradients():
    """Residual actions from v0 = 0 give the CG iterates (Sec. 3.2, Hestenes & Stiefel)."""
    K, Khat, b, kmv, winv = _system()
    NC = b.size
    iterates = []
    O.itergp(kmv, winv, b, np.zeros((NC, 0)), np.zeros((NC, 0)), policy=O.CG,
             max_iters=8, tol_abs=0, tol_rel=0,
             on_iterate=lambda j, v, Q: iterates.append(v.copy()))
    ref = textbook_cg(Khat, b, 8)
    for a, r in zip(iterates, ref):
        assert np.allclose(a, r, rtol=1e-8, atol=1e-10)


def test_iterates_match_eq11_projection_and_root_is_khat_orthonormal():
    """v_j = S_j (S_j^T K_hat S_j)^-1 S_j^T b (Eq. 11) for the actions taken; Q^T K_hat Q = I;
    the marginal variance is non-increasing in j (Prop. A.3)."""
    K, Khat, b, kmv, winv = _system(n=8)
    NC = b.size
    seen = []
    v, Q, S, T, info = O.itergp(kmv, winv, b, np.zeros((NC, 0)), np.zeros((NC, 0)),
                                policy=O.CG, max_iters=10, tol_abs=0, tol_rel=0,
                                on_iterate=lambda j, v, Q: seen.append((v.copy(), Q.copy())))
    Sj = S
    Cj = Sj @ np.linalg.solve(Sj.T @ Khat @ Sj, Sj.T)
    assert np.allclose(v, Cj @ b, rtol=1e-8, atol=1e-10)
    assert np.allclose(Q.T @ Khat @ Q, np.eye(Q.shape[1]), atol=1e-8)
    assert np.allclose(T, K @ S, atol=1e-12)
    kx = K[:6]                       # covariances of 2 training points' outputs with all
    prev = None
    for _, Qj in seen:
        var = np.diag(K[:6, :6]) - np.sum((kx @ Qj) ** 2, axis=1)
        if prev is not None:
            assert np.all(var <= prev + 1e-12)
        prev = var


# ---------------------------------------------------------------------- Alg. 3

def test_virtual_solver_run_projected_residual_and_error_vanish():
    """After the virtual run, S^T r0 = 0 (Prop. A.4) and C0 K_hat (v* - v0) = 0 (Prop. A.5)."""
    K, Khat, b, kmv, winv = _system()
    NC = b.size
    g = np.random.default_rng(2)
    S = g.standard_normal((NC, 6))
    T = K @ S
    winv_cols = lambda M: np.stack([winv(M[:, k]) for k in range(M.shape[1])], axis=1)
    Q0, S2, T2, dropped = O.virtual_solver_run(S, T, winv_cols, R=None)
    v0 = Q0 @ (Q0.T @ b)
    r0 = b - Khat @ v0
    assert dropped == 0
    assert np.allclose(S.T @ r0, 0.0, atol=1e-9 * np.linalg.norm(b))
    vstar = np.linalg.solve(Khat, b)
    assert np.allclose(Q0 @ (Q0.T @ (Khat @ (vstar - v0))), 0.0, atol=1e-9)
    # C0 = S (S^T K_hat S)^-1 S^T (Eq. 12) independent of the rotation
    C0 = S @ np.linalg.solve(S.T @ Khat @ S, S.T)
    assert np.allclose(Q0 @ Q0.T, C0, atol=1e-10)
    assert np.allclose(T2, K @ S2, atol=1e-10)


def test_compression_rank_limits():
    """R >= rank reproduces the uncompressed run; R = 0 equals no recycling (Fig. 4)."""
    X, y, kern = tiny_problem(n=10, ell=0.7)
    lik = O.Softmax(y, 3)
    kw = dict(max_newton=3, max_iters=6, tol_abs=0, tol_rel=0)
    full = O.iterncgp_fit(X, lik, 3, kern, R=None, **kw)
    big = O.iterncgp_fit(X, lik, 3, kern, R=1000, **kw)
    zero = O.iterncgp_fit(X, lik, 3, kern, R=0, **kw)
    norec = O.iterncgp_fit(X, lik, 3, kern, recycle=False, **kw)
    assert np.allclose(full.f, big.f, atol=1e-12)
    assert np.allclose(zero.f, norec.f, atol=1e-12)
    assert not np.allclose(full.f, norec.f, atol=1e-6)


def test_trace_identity_with_eigenvector_actions():
    """Prop. A.6: with W^-1 = 0 and actions = eigenvectors of K, Tr K_{i,0} = Tr K - Tr M."""
    X, _, kern = tiny_problem(n=9, ell=0.8)
    K = O.dense_K(X, 2, kern)
    lam, V = np.linalg.eigh(K)
    S = V[:, -5:]
    Q0, S2, T2, _ = O.virtual_solver_run(S, K @ S, lambda M: 0 * M, R=None)
    M = S.T @ (K @ S)
    lhs = np.trace(K) - np.trace(K @ (Q0 @ Q0.T) @ K)
    assert lhs == pytest.approx(np.trace(K) - np.trace(M), rel=1e-10)
    assert lhs == pytest.approx(lam[:-5].sum(), rel=1e-8)


def test_truncation_keeps_largest_eigenpairs():
    K, Khat, b, kmv, winv = _system()
    NC = b.size
    S = np.random.default_rng(4).standard_normal((NC, 7))
    winv_cols = lambda M: np.stack([winv(M[:, k]) for k in range(M.shape[1])], axis=1)
    Q0, S2, T2, _ = O.virtual_solver_run(S, K @ S, winv_cols, R=3)
    M = S.T @ (Khat @ S)
    lam = np.sort(np.linalg.eigvalsh(0.5 * (M + M.T)))[::-1]
    M2 = S2.T @ (Khat @ S2)
    assert np.allclose(M2, np.diag(lam[:3]), atol=1e-8 * lam[0])
    assert S2.shape[1] == 3 and Q0.shape[1] == 3


# ---------------------------------------------------------------------- Alg. 1

def test_gaussian_likelihood_converges_in_one_newton_step():
    """Thm. A.2: Gaussian likelihood -> pseudo targets = y, f_1 = f_MAP (= f_2)."""
    X, _, kern = tiny_problem(n=10)
    yr = np.random.default_rng(3).standard_normal((10, 1))
    lik = O.Gaussian(yr, noise=0.3)
    f0 = np.random.default_rng(4).standard_normal((10, 1))
    assert np.allclose(O.pseudo_targets(lik, f0), yr, atol=1e-14)
    res = O.iterncgp_fit(X, lik, 1, kern, max_newton=3, max_iters=10, tol_abs=0, tol_rel=0)
    assert np.allclose(res.fs[1], res.fs[2], atol=1e-9)
    k = O.kernel_matrix(X, X, kern)
    fmap = k @ np.linalg.solve(k + 0.3 * np.eye(10), yr)     # GP regression posterior mean
    assert np.allclose(res.fs[1], fmap, atol=1e-9)


@pytest.mark.parametrize("recycle", [True, False])
def test_converged_solves_track_exact_newton(recycle):
    """With enough CG iterations per step, Alg. 1 reproduces the exact Newton iterates."""
    X, y, kern = tiny_problem(n=10, ell=0.7)
    lik = O.Softmax(y, 3)
    ex, _ = O.exact_newton(X, lik, 3, kern, steps=4)
    res = O.iterncgp_fit(X, lik, 3, kern, max_newton=4, max_iters=30, tol_abs=1e-12,
                         tol_rel=1e-12, recycle=recycle)
    for a, b_ in zip(res.fs, ex):
        assert np.allclose(a, b_, rtol=1e-7, atol=1e-8)


# ---------------------------------------------------------------------- predictive

def test_predictive_with_unit_actions_equals_literal_eq5():
    X, y, kern = tiny_problem(n=8, ell=0.6)
    C = 3
    lik = O.Softmax(y, C)
    Xs = datagen.blobs(5, 2, 3, 99)[0]
    res = O.iterncgp_fit(X, lik, C, kern, max_newton=1, max_iters=8 * C, policy=O.UNIT,
                         tol_abs=0, tol_rel=0)
    mean, var, probs = O.predict(Xs, X, res.v, res.Q, kern, C)
    em, ev = O.exact_predict(Xs, X, lik, res.fs[0], res.fs[1], kern, C, contrasts_only=False)
    assert np.allclose(mean, em, atol=1e-8)
    assert np.allclose(var, ev, atol=1e-8)
    assert np.allclose(probs.sum(axis=1), 1.0)


def test_predictive_with_converged_cg_matches_mean_and_bounds_variance():
    """Converged CG reproduces the Laplace mean (Eq. 9 vs Eq. 4); its Krylov actions stay
    in the class-contrast subspace, so C_j <= K_hat^-1 restricted there and the variance
    is bounded below by the contrasts-only Laplace variance (and above by s)."""
    X, y, kern = tiny_problem(n=8, ell=0.6)
    C = 3
    lik = O.Softmax(y, C)
    Xs = datagen.blobs(5, 2, 3, 99)[0]
    res = O.iterncgp_fit(X, lik, C, kern, max_newton=2, max_iters=8 * (C - 1),
                         tol_abs=1e-13, tol_rel=1e-13, recycle=False)
    mean, var, _ = O.predict(Xs, X, res.v, res.Q, kern, C)
    em, ev = O.exact_predict(Xs, X, lik, res.fs[1], res.fs[2], kern, C, contrasts_only=True)
    assert np.allclose(mean, em, atol=1e-7)
    assert np.all(var >= ev - 1e-7)
    assert np.all(var <= kern.outputscale + 1e-12)


def test_predictive_variance_is_non_increasing_in_the_iterations():
    """The predictive function's marginal variance (Eq. 10) shrinks with every IterGP
    iteration (Prop. A.3: C_j grows by the PSD term d_j d_j^T / eta_j).  With an empty
    buffer the root Q gains one column per iteration, so the variance after j iterations
    uses its first j columns; it starts at the prior s, never increases, and ends strictly
    below s at test points next to training points."""
    X, y, kern = tiny_problem(n=10, ell=0.8)
    C = 3
    res = O.iterncgp_fit(X, O.Softmax(y, C), C, kern, max_newton=1, max_iters=12,
                         tol_abs=0, tol_rel=0, recycle=False)
    assert res.Q.shape[1] == res.infos[0].iters == 12
    Xs = np.concatenate([X[:3] + 0.05, datagen.blobs(4, 2, 3, 98)[0]])
    prev = None
    for j in range(res.Q.shape[1] + 1):
        _, var, _ = O.predict(Xs, X, res.v, res.Q[:, :j], kern, C)
        if j == 0:
            assert np.allclose(var, kern.outputscale)
        else:
            assert np.all(var <= prev + 1e-12)
        prev = var
    assert np.all(prev[:3] < kern.outputscale - 1e-3)


def test_predictive_with_contrast_spanning_actions_equals_laplace_predictive():
    """A virtual solver run over actions spanning range(I kron P) (dependent columns are
    dropped as zero eigenpairs) gives C0 = K_hat^-1 restricted to the class contrasts,
    i.e. the Laplace predictive with W singular (Eqs. 4-5)."""
    X, y, kern = tiny_problem(n=7, ell=0.6)
    C, N = 3, 7
    lik = O.Softmax(y, C)
    f = np.random.default_rng(11).standard_normal((N, C))
    f -= f.mean(axis=1, keepdims=True)
    K = O.dense_K(X, C, kern)
    Pi = np.kron(np.eye(N), np.eye(C) - np.ones((C, C)) / C)
    S = Pi.copy()
    winv_cols = lambda M: np.stack([lik.Winv_apply(f, M[:, k].reshape(N, C)).reshape(-1)
                                    for k in range(M.shape[1])], axis=1)
    Q0, S2, _, dropped = O.virtual_solver_run(S, K @ S, winv_cols, R=None, drop_rel=1e-10)
    assert S2.shape[1] == N * (C - 1) and dropped == N
    b = O.pseudo_targets(lik, f).reshape(-1)
    v = (Q0 @ (Q0.T @ b)).reshape(N, C)
    f_next = (K @ v.reshape(-1)).reshape(N, C)
    Xs = datagen.blobs(4, 2, 3, 5)[0]
    mean, var, _ = O.predict(Xs, X, v, Q0, kern, C)
    em, ev = O.exact_predict(Xs, X, lik, f, f_next, kern, C, contrasts_only=True)
    assert np.allclose(mean, em, atol=1e-7)
    assert np.allclose(var, ev, atol=1e-8)
    vN, _ = O.exact_newton_step(X, lik, f, np.zeros((N, C)), kern)
    assert np.allclose(v, vN, atol=1e-8)


def test_probit_reduces_to_softmax_at_zero_variance():
    X, y, kern = tiny_problem(n=6)
    v = np.random.default_rng(1).standard_normal((6, 3))
    Xs = X[:3]
    mean, var, probs = O.predict(Xs, X, v, np.zeros((18, 0)), kern, 3)
    assert np.allclose(var, kern.outputscale)
    assert np.allclose(probs, O.softmax(mean / math.sqrt(1 + math.pi / 8 * kern.outputscale)))


def test_class_contrast_projection_is_the_identity_in_exact_arithmetic():
    """The CUDA path removes the per-point class mean from y_hat - m and from each residual.
    Both lie in range(I kron P) in exact arithmetic (f = K v with v there; W^+ maps into it,
    Lemma A.6), so in FP64 the projected and the literal runs coincide."""
    X, y, _ = datagen.blobs(60, 2, 3, 21)
    kern = O.Kernel(O.RBF, 1.0, 1.0)
    lik = O.Softmax(y, 3)
    kw = dict(max_newton=6, max_iters=10, R=15, tol_abs=0, tol_rel=0)
    a = O.iterncgp_fit(X, lik, 3, kern, **kw)
    b = O.iterncgp_fit(X, lik, 3, kern, project_contrasts=True, **kw)
    for fa, fb in zip(a.fs, b.fs):
        assert np.allclose(fa, fb, rtol=1e-8, atol=1e-9)
    assert np.allclose(a.v.sum(axis=1), 0.0, atol=1e-8)


def test_restart_from_an_iterate_reproduces_the_next_step():
    """Without recycling a Newton step depends only on f_i (Alg. 1), so restarting the fit
    at its own iterate f_i reproduces f_{i+1}; pins the starting-iterate option that the
    teacher-forced GPU tests use."""
    X, y, _, _ = datagen.workload_small(n_train=120, n_test=2)
    kern = O.Kernel(O.RBF, 1.0, 1.0)
    full = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, max_newton=4, max_iters=8, recycle=False,
                          tol_abs=0, tol_rel=0)
    for i in range(3):
        step = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, max_newton=1, max_iters=8,
                              recycle=False, tol_abs=0, tol_rel=0, f0=full.fs[i])
        assert np.allclose(step.f, full.fs[i + 1], rtol=0, atol=1e-12 * np.abs(full.fs[i + 1]).max())


def test_product_noise_off_is_the_exact_fit_and_enters_each_product_linearly():
    """The inexact-product option that the batched GPU tests use to measure a fit's
    sensitivity to rounding.  eps = 0 is bitwise the exact fit; every kernel product draws
    its own noise (Alg. 2 as the oracle runs it: K v for the residual r_{j-1} and K s_j per
    iteration, then f = K v once per Newton step, Alg. 1); and for a small eps the fit moves
    linearly in eps (the same draws at 2 eps move it twice as far)."""
    X, y, _ = datagen.blobs(60, 2, 3, 21)
    kern = O.Kernel(O.RBF, 1.0, 1.0)
    kw = dict(max_newton=3, max_iters=5, R=10, tol_abs=0, tol_rel=0)
    exact = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, **kw)
    zero = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, product_noise=(0.0, np.random.default_rng(1)), **kw)
    assert np.array_equal(exact.f, zero.f)

    class Counting:
        def __init__(self, seed):
            self.g, self.calls = np.random.default_rng(seed), 0

        def standard_normal(self, shape):
            self.calls += 1
            return self.g.standard_normal(shape)

    rng = Counting(0)
    res = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, product_noise=(1e-8, rng), **kw)
    assert rng.calls == sum(2 * inf.iters + 1 for inf in res.infos) == 33

    d1 = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, product_noise=(1e-8, np.random.default_rng(1)), **kw).f - exact.f
    d2 = O.iterncgp_fit(X, O.Softmax(y, 3), 3, kern, product_noise=(2e-8, np.random.default_rng(1)), **kw).f - exact.f
    assert 0 < np.linalg.norm(d1) <= 1e-6 * np.linalg.norm(exact.f)
    assert np.linalg.norm(d2 - 2.0 * d1) <= 1e-3 * np.linalg.norm(d2)


# ------------------------------------------------------ one-latent likelihoods (App. A, C)

def one_latent_problem(kind, n=12, seed=3):
    g = np.random.default_rng(seed)
    X = g.uniform(-2, 2, size=(n, 2))
    ftrue = np.sin(X[:, 0]) + 0.5 * X[:, 1]
    if kind == "bernoulli":
        y = (g.random(n) < 1 / (1 + np.exp(-2 * ftrue))).astype(np.int64)
        lik = O.Bernoulli(y)
    else:
        y = g.poisson(np.exp(ftrue))
        lik = O.Poisson(y)
    return X, y, lik


@pytest.mark.parametrize("kind", ["bernoulli", "poisson"])
def test_one_latent_loglik_against_scipy_pmfs(kind):
    X, y, lik = one_latent_problem(kind)
    f = np.random.default_rng(4).standard_normal((len(y), 1))
    if kind == "bernoulli":
        ref = scipy.stats.bernoulli.logpmf(y, scipy.special.expit(f[:, 0])).sum()
    else:   # the oracle drops the constant -log y!
        ref = scipy.stats.poisson.logpmf(y, np.exp(f[:, 0])).sum() + scipy.special.gammaln(y + 1.0).sum()
    assert np.isclose(lik.loglik(f), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["bernoulli", "poisson"])
def test_one_latent_gradient_and_hessian_by_finite_differences(kind):
    X, y, lik = one_latent_problem(kind)
    f = np.random.default_rng(5).standard_normal((len(y), 1))
    h = 1e-5
    for i in range(len(y)):
        e = np.zeros_like(f)
        e[i] = h
        g_fd = (lik.loglik(f + e) - lik.loglik(f - e)) / (2 * h)
        assert np.isclose(lik.grad(f)[i, 0], g_fd, rtol=1e-6, atol=1e-8)
        hess_fd = (lik.grad(f + e)[i, 0] - lik.grad(f - e)[i, 0]) / (2 * h)
        assert np.isclose(lik.winv_diag(f)[i, 0], -1.0 / hess_fd, rtol=1e-6)


def textbook_newton_diag(K, w, grad, f, m):
    """Eq. 3 with a diagonal W = diag(w): f + (W + K^-1)^-1 (grad - K^-1 (f - m))."""
    Kinv = np.linalg.inv(K)
    g = grad.reshape(-1) - Kinv @ (f - m).reshape(-1)
    return f + np.linalg.solve(np.diag(w) + Kinv, g).reshape(f.shape)


@pytest.mark.parametrize("kind", ["bernoulli", "poisson"])
def test_one_latent_newton_via_pseudo_targets_equals_textbook_newton(kind):
    """Alg. 1's GP-regression form of the step (pseudo targets, noise W^-1; shift 0 for a
    single latent) equals Eq. 3 with W from a finite-difference Hessian."""
    X, y, lik = one_latent_problem(kind)
    kern = O.Kernel(O.RBF, 0.8, 1.0)
    K = O.kernel_matrix(X, X, kern)
    m = np.zeros((len(y), 1))
    f = m.copy()
    h = 1e-5
    for _ in range(4):
        _, f_next = O.exact_newton_step(X, lik, f, m, kern, shift=0.0)
        w = np.array([-(lik.grad(f + h * np.eye(len(y))[:, [i]])[i, 0]
                        - lik.grad(f - h * np.eye(len(y))[:, [i]])[i, 0]) / (2 * h)
                      for i in range(len(y))])
        ref = textbook_newton_diag(K, w, lik.grad(f), f, m)
        assert np.allclose(f_next, ref, rtol=1e-6, atol=1e-7)
        f = f_next
    # at the mode grad log p = K^-1 (f - m) = v (Eq. 3)
    fs, vs = O.exact_newton(X, lik, 1, kern, steps=15, shift=0.0)
    assert np.allclose(lik.grad(fs[-1]), vs[-1], atol=1e-8)


@pytest.mark.parametrize("kind", ["bernoulli", "poisson"])
def test_one_latent_unit_actions_reproduce_the_exact_step(kind):
    """N unit-vector actions (C = 1) reproduce the exact Newton step (Alg. 2 / Sec. 3)."""
    X, y, lik = one_latent_problem(kind, n=10)
    kern = O.Kernel(O.RBF, 0.8, 1.0)
    ref = O.exact_newton(X, lik, 1, kern, steps=3, shift=0.0)[0]
    res = O.iterncgp_fit(X, lik, 1, kern, max_newton=3, max_iters=len(y), policy=O.UNIT,
                         recycle=False, tol_abs=0, tol_rel=0)
    for a, b in zip(res.fs, ref):
        assert np.allclose(a, b, atol=1e-9)


# ---------------------------------------------------------------------- one kernel per class

def class_kernels(C=3):
    """Distinct hyperparameters (and kinds) per output GP."""
    table = [(O.RBF, 0.5, 1.3), (O.MATERN32, 0.9, 0.7), (O.RBF, 1.6, 2.1), (O.MATERN32, 0.35, 1.0)]
    return O.ClassKernels(tuple(O.Kernel(*table[c]) for c in range(C)))


def test_class_kernel_product_brute_force_double_loop():
    """Y[i, j] = sum_n k_{j mod C}(a_i, b_n) S[n, j], evaluated term by term."""
    g = np.random.default_rng(5)
    C = 3
    A, B = g.standard_normal((6, 3)), g.standard_normal((9, 3))
    S = g.standard_normal((9, 2 * C))
    kerns = class_kernels(C)
    Y = np.zeros((6, 2 * C))
    for i in range(6):
        for n in range(9):
            r = math.sqrt(sum((A[i, d] - B[n, d]) ** 2 for d in range(3)))
            for j in range(2 * C):
                kc = kerns.kernels[j % C]
                u = r / kc.lengthscale
                if kc.kind == O.RBF:
                    k = kc.outputscale * math.exp(-u * u / 2)
                else:
                    k = kc.outputscale * (1 + math.sqrt(3) * u) * math.exp(-math.sqrt(3) * u)
                Y[i, j] += k * S[n, j]
    assert np.allclose(O.kmatvec_classes(A, B, S, kerns, C), Y, rtol=1e-12, atol=1e-12)


def test_class_kernel_prior_is_block_diagonal_per_class():
    """CN ordering: entry (n C + c, m C + e) = k_c(x_n, x_m) delta_ce; the matrix-free
    product of a stacked NC-vector equals the dense matrix times it."""
    X, _, _ = tiny_problem(n=5)
    C = 3
    kerns = class_kernels(C)
    K = O.dense_K(X, C, kerns)
    for c, kc in enumerate(kerns.kernels):
        kx = O.kernel_matrix(X, X, kc)
        for n in range(5):
            for m in range(5):
                blk = K[n * C:(n + 1) * C, m * C:(m + 1) * C]
                assert blk[c, c] == pytest.approx(kx[n, m], rel=1e-12)
                assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
    w = np.random.default_rng(2).standard_normal((5, C))
    assert np.allclose(O.kmatvec_classes(X, X, w, kerns, C).reshape(-1), K @ w.reshape(-1), atol=1e-12)


def test_class_kernel_step_with_invertible_w_equals_textbook_newton():
    """With an invertible W (Gaussian likelihood over C outputs, W^-1 = sigma^2 I) the
    pseudo-target step of Eqs. 6-7 is Newton's step (Eq. 3) for any prior, so also for one
    kernel per output; one step reaches the posterior mean."""
    X, _, _ = tiny_problem(n=9, ell=0.6)
    C = 3
    kerns = class_kernels(C)
    yr = np.random.default_rng(8).standard_normal((9, C))
    lik = O.Gaussian(yr, 0.3)
    K = O.dense_K(X, C, kerns)
    m = np.zeros((9, C))
    f = np.random.default_rng(9).standard_normal((9, C))
    _, f_next = O.exact_newton_step(X, lik, f, m, kerns, shift=0.0)
    W = np.eye(9 * C) / 0.3
    Kinv = np.linalg.inv(K)
    g = lik.grad(f).reshape(-1) - Kinv @ f.reshape(-1)
    ref = f + np.linalg.solve(W + Kinv, g).reshape(9, C)
    assert np.allclose(f_next, ref, rtol=1e-8, atol=1e-9)
    post = (K @ np.linalg.solve(K + 0.3 * np.eye(9 * C), yr.reshape(-1))).reshape(9, C)
    assert np.allclose(f_next, post, rtol=1e-8, atol=1e-9)


def test_class_kernel_softmax_fixed_point_of_the_pseudo_inverse_iteration():
    """Under softmax, W^+ (footnote to Eq. 6) vanishes on the per-point class sums.  A
    fixed point f = K v + m of the pseudo-target step then satisfies W^+ (v - grad log p)
    = 0: v agrees with the gradient on the class contrasts.  With one shared kernel K keeps
    the class sums invariant and the fixed point is the mode (v = grad); with distinct
    kernels it is not, and its objective (Eq. 2) stays below the mode's."""
    X, y, _ = tiny_problem(n=9, ell=0.6)
    C = 3
    kerns = class_kernels(C)
    lik = O.Softmax(y, C)
    K = O.dense_K(X, C, kerns)
    fs, vs = O.exact_newton(X, lik, C, kerns, steps=40)
    f, v = fs[-1], vs[-1]
    g = lik.grad(f)
    contrast = lambda a: a - a.mean(axis=1, keepdims=True)
    assert np.allclose(contrast(v), contrast(g), atol=1e-9)
    assert np.allclose(f, (K @ v.reshape(-1)).reshape(9, C), atol=1e-12)
    # the mode of Eq. 2 under the same prior (textbook Newton, Eq. 3)
    fm = np.zeros((9, C))
    for _ in range(40):
        fm = textbook_newton_step(K, lik, fm, np.zeros((9, C)))
    psi = lambda a: lik.loglik(a) - 0.5 * a.reshape(-1) @ np.linalg.solve(K, a.reshape(-1))
    assert np.allclose(lik.grad(fm).reshape(-1), np.linalg.solve(K, fm.reshape(-1)), atol=1e-10)
    assert psi(f) < psi(fm)
    assert np.abs(v.sum(axis=1)).max() > 1e-3           # the class sums of v are not zero


def test_class_kernel_unit_actions_reproduce_the_exact_step():
    """With NC unit-vector actions IterGP is a direct solve: the fit's f_1 is the exact
    Newton step under the per-class prior."""
    X, y, _ = tiny_problem(n=8, ell=0.6)
    C = 3
    kerns = class_kernels(C)
    lik = O.Softmax(y, C)
    res = O.iterncgp_fit(X, lik, C, kerns, max_newton=2, max_iters=8 * C, policy=O.UNIT,
                         tol_abs=0, tol_rel=0, recycle=False)
    fs, _ = O.exact_newton(X, lik, C, kerns, steps=2)
    assert np.allclose(res.fs[1], fs[1], rtol=1e-8, atol=1e-9)
    assert np.allclose(res.fs[2], fs[2], rtol=1e-7, atol=1e-8)


def test_class_kernel_predictive_with_unit_actions_equals_literal_eq5():
    X, y, _ = tiny_problem(n=8, ell=0.6)
    C = 3
    kerns = class_kernels(C)
    lik = O.Softmax(y, C)
    Xs = datagen.blobs(5, 2, 3, 99)[0]
    res = O.iterncgp_fit(X, lik, C, kerns, max_newton=1, max_iters=8 * C, policy=O.UNIT,
                         tol_abs=0, tol_rel=0)
    mean, var, probs = O.predict(Xs, X, res.v, res.Q, kerns, C)
    em, ev = O.exact_predict(Xs, X, lik, res.fs[0], res.fs[1], kerns, C, contrasts_only=False)
    assert np.allclose(mean, em, atol=1e-8)
    assert np.allclose(var, ev, atol=1e-8)
    # the prior variance of class c is its own outputscale
    far = np.full((1, 2), 1e3)
    _, vfar, _ = O.predict(far, X, res.v, res.Q, kerns, C)
    assert np.allclose(vfar[0], [k.outputscale for k in kerns.kernels])


def test_equal_class_kernels_reduce_to_the_shared_kernel():
    X, y, kern = tiny_problem(n=14, ell=0.8)
    C = 3
    lik = O.Softmax(y, C)
    a = O.iterncgp_fit(X, lik, C, kern, max_newton=3, max_iters=6, R=8)
    b = O.iterncgp_fit(X, lik, C, O.ClassKernels((kern,) * C), max_newton=3, max_iters=6, R=8)
    assert np.allclose(a.f, b.f, rtol=1e-10, atol=1e-12)
    assert np.allclose(a.v, b.v, rtol=1e-10, atol=1e-12)
    Xs = datagen.blobs(6, 2, 3, 4)[0]
    for u, w in zip(O.predict(Xs, X, a.v, a.Q, kern, C), O.predict(Xs, X, b.v, b.Q, O.ClassKernels((kern,) * C), C)):
        assert np.allclose(u, w, rtol=1e-10, atol=1e-12)
