"""Property-based pins of the oracle (host only): the identities the fixed-seed pins check,
over random shapes, class counts, logits and kernels.  Each property is fixed by the
mathematics, not by the oracle's own formulas."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle.itergp_oracle as O

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

# derandomized: the same examples on every run, so a rare ill-conditioned draw cannot make
# the suite flaky
SETTINGS = settings(max_examples=30, deadline=None, derandomize=True)


@SETTINGS
@given(n=st.integers(1, 6), c=st.integers(2, 6), scale=st.floats(0.1, 6.0), seed=st.integers(0, 2**31 - 1))
def test_w_pseudo_inverse_is_moore_penrose(n, c, scale, seed):
    """Lemma A.6 at random logits: P diag(1/pi) P is the Moore-Penrose inverse of each
    softmax Hessian block, W W^+ = P, and W^+ 1 = 0."""
    g = np.random.default_rng(seed)
    f = scale * g.standard_normal((n, c))
    lik = O.Softmax(g.integers(0, c, n), c)
    Wb = lik.W_blocks(f)
    Wd = lik.Winv_dense(f)
    P = np.eye(c) - np.ones((c, c)) / c
    for k in range(n):
        A, Ap = Wb[k], Wd[k * c:(k + 1) * c, k * c:(k + 1) * c]
        assert np.allclose(A @ Ap @ A, A, atol=1e-10 * max(1.0, np.abs(A).max()))
        assert np.allclose(A @ Ap, P, atol=1e-9)
        assert np.allclose(A.sum(axis=1), 0.0, atol=1e-12)      # rows of W sum to zero
    assert np.allclose(lik.Winv_apply(f, np.ones((n, c))), 0.0, atol=1e-9)


@SETTINGS
@given(m=st.integers(1, 7), n=st.integers(1, 7), d=st.integers(1, 5), p=st.integers(1, 4),
       kind=st.sampled_from([O.RBF, O.MATERN32]), ell=st.floats(0.2, 5.0), s=st.floats(0.1, 3.0),
       seed=st.integers(0, 2**31 - 1))
def test_kernel_product_equals_the_double_loop(m, n, d, p, kind, ell, s, seed):
    """k(A, B) S against a double loop over the textbook kernel formulas on scipy's
    Euclidean distances."""
    g = np.random.default_rng(seed)
    A, B, S = g.standard_normal((m, d)), g.standard_normal((n, d)), g.standard_normal((n, p))
    r = cdist(A, B)
    want = np.zeros((m, p))
    for i in range(m):
        for j in range(n):
            if kind == O.RBF:
                k = s * np.exp(-r[i, j] ** 2 / (2 * ell ** 2))
            else:
                z = np.sqrt(3.0) * r[i, j] / ell
                k = s * (1 + z) * np.exp(-z)
            want[i] += k * S[j]
    got = O.kmatvec(A, B, S, O.Kernel(kind, ell, s))
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12)


@SETTINGS
@given(n=st.integers(2, 8), d=st.integers(1, 4), kind=st.sampled_from([O.RBF, O.MATERN32]),
       ell=st.floats(0.3, 3.0), seed=st.integers(0, 2**31 - 1))
def test_kernel_matrix_is_symmetric_psd_with_the_outputscale_on_its_diagonal(n, d, kind, ell, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, d))
    K = O.kernel_matrix(X, X, O.Kernel(kind, ell, 1.7))
    assert np.allclose(K, K.T, atol=1e-14)
    assert np.allclose(np.diag(K), 1.7, atol=1e-12)
    assert np.linalg.eigvalsh(K).min() >= -1e-10 * 1.7


@SETTINGS
@given(n=st.integers(1, 6), c=st.integers(2, 6), seed=st.integers(0, 2**31 - 1))
def test_softmax_gradient_sums_to_zero_and_pseudo_targets_stay_in_the_contrasts(n, c, seed):
    """sum_c grad_c = 0 per point, so W^+ grad and y_hat - f have zero class mean."""
    g = np.random.default_rng(seed)
    f = 2 * g.standard_normal((n, c))
    lik = O.Softmax(g.integers(0, c, n), c)
    assert np.allclose(lik.grad(f).sum(axis=1), 0.0, atol=1e-12)
    yhat = O.pseudo_targets(lik, f)
    assert np.allclose((yhat - f).sum(axis=1), 0.0, atol=1e-9)


def _random_system(n, c, seed, ell):
    """A tiny softmax Newton system K_hat v = b at random logits (exact K_hat, dense)."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, 2))
    kern = O.Kernel(O.RBF, ell, 1.0)
    lik = O.Softmax(g.integers(0, c, n), c)
    f = g.standard_normal((n, c))
    f -= f.mean(axis=1, keepdims=True)
    K = O.dense_K(X, c, kern)
    Khat = K + lik.Winv_dense(f)
    b = O.pseudo_targets(lik, f).reshape(-1)
    kmv = lambda w: K @ w                                              # noqa: E731
    winv = lambda w: lik.Winv_apply(f, w.reshape(n, c)).reshape(-1)    # noqa: E731
    return Khat, b, kmv, winv


@SETTINGS
@given(n=st.integers(1, 4), c=st.integers(2, 3), seed=st.integers(0, 2**31 - 1))
def test_nc_unit_actions_reproduce_the_direct_solve(n, c, seed):
    """Sec. 3.2 / Eq. 11: NC unit-vector actions span R^NC, so v = K_hat^-1 b and
    Q Q^T = K_hat^-1 (well-conditioned: short lengthscale, so K_hat ~ I + W^+)."""
    Khat, b, kmv, winv = _random_system(n, c, seed, ell=0.3)
    NC = b.size
    v, Q, _, _, info = O.itergp(kmv, winv, b, np.zeros((NC, 0)), np.zeros((NC, 0)),
                                policy=O.UNIT, max_iters=NC, tol_abs=0, tol_rel=0)
    assert info.iters == NC
    assert np.allclose(v, np.linalg.solve(Khat, b), rtol=1e-8, atol=1e-9)
    assert np.allclose(Q @ Q.T, np.linalg.inv(Khat), rtol=1e-6, atol=1e-8)


@SETTINGS
@given(n=st.integers(2, 6), c=st.integers(2, 4), iters=st.integers(1, 6), seed=st.integers(0, 2**31 - 1))
def test_the_root_stays_khat_orthonormal(n, c, iters, seed):
    """Alg. 2 builds Q with Q^T K_hat Q = I (C_j K_hat C_j = C_j) for any number of CG
    iterations, including when it stops early on eta <= 0 or a zero residual."""
    Khat, b, kmv, winv = _random_system(n, c, seed, ell=0.8)
    NC = b.size
    v, Q, _, _, info = O.itergp(kmv, winv, b, np.zeros((NC, 0)), np.zeros((NC, 0)),
                                policy=O.CG, max_iters=iters, tol_abs=0, tol_rel=0)
    assert np.allclose(Q.T @ Khat @ Q, np.eye(Q.shape[1]), atol=1e-7)
    assert np.allclose(v, Q @ (Q.T @ b), rtol=1e-8, atol=1e-9)   # v_j = C_j b from v_0 = 0


@SETTINGS
@given(n=st.integers(2, 5), c=st.integers(2, 3), k=st.integers(1, 5), seed=st.integers(0, 2**31 - 1))
def test_virtual_solver_run_projects_out_the_recycled_actions(n, c, k, seed):
    """Alg. 3 on k random recycled actions (k <= NC): S^T r_0 = 0 (Prop. A.4), the
    recycled root equals S (S^T K_hat S)^-1 S^T (Eq. 12) and T stays K S."""
    Khat, b, kmv, winv = _random_system(n, c, seed, ell=0.5)
    NC = b.size
    k = min(k, NC)
    S = np.random.default_rng(seed + 1).standard_normal((NC, k))
    T = np.stack([kmv(S[:, j]) for j in range(k)], axis=1)
    winv_cols = lambda M: np.stack([winv(M[:, j]) for j in range(M.shape[1])], axis=1)  # noqa: E731
    Q0, S2, T2, dropped = O.virtual_solver_run(S, T, winv_cols, R=None)
    assert dropped == 0
    v0 = Q0 @ (Q0.T @ b)
    assert np.allclose(S.T @ (b - Khat @ v0), 0.0, atol=1e-8 * np.linalg.norm(b))
    assert np.allclose(Q0 @ Q0.T, S @ np.linalg.solve(S.T @ Khat @ S, S.T), atol=1e-8)
    assert np.allclose(T2, np.stack([kmv(S2[:, j]) for j in range(S2.shape[1])], axis=1), atol=1e-10)
