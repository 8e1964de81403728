"""How far rounding of a kernel product's size moves the oracle's own fit (Alg. 1-2, CG
actions): the evidence behind the batched parity tests' rounding band.  CPU only."""
import numpy as np

import oracle.itergp_oracle as O
from paper_2310_20285_gb300 import datagen

SPLIT_EPS = 2.0 ** -21   # relative rounding of one term of the split (FP16 hi/lo) product


def band(p, eps, seeds=8):
    kern = O.Kernel(O.RBF, p.lengthscale, 1.0)
    X = p.X.astype(np.float64)
    kw = dict(max_newton=3, max_iters=6, R=10, tol_abs=0.0, tol_rel=0.0)
    ref = O.iterncgp_fit(X, O.Softmax(p.y, p.c), p.c, kern, **kw)
    em, _, _ = O.predict(p.Xs.astype(np.float64), X, ref.v, ref.Q, kern, p.c)
    errs = []
    for seed in range(seeds):
        r = O.iterncgp_fit(X, O.Softmax(p.y, p.c), p.c, kern,
                           product_noise=(eps, np.random.default_rng(seed)), **kw)
        mean, _, _ = O.predict(p.Xs.astype(np.float64), X, r.v, r.Q, kern, p.c)
        errs.append(np.linalg.norm(mean - em) / np.linalg.norm(em))
    return np.array(errs)


def test_the_smooth_2d_problem_amplifies_product_rounding_past_the_bar():
    """The batched tests' small batch (seed 41): its smooth 2-D problem (N = 576, C = 4,
    l = 1.82) moves by more than the 1e-4 bar under rounding of the split product's size,
    even at the median of the draws, while a 2-D problem of the same batch with a shorter
    lengthscale (N = 828, l = 1.16) stays two orders of magnitude inside it.  Halving the
    rounding halves the spread (the response is linear), so the band measures the
    problem's sensitivity, not the draws."""
    probs = datagen.batch_problems(count=7, seed=41, n_lo=150, n_hi=1400, dims=(2, 5, 8, 16),
                                   c_lo=2, c_hi=7, ell_lo=0.8, ell_hi=3.0, n_test=40)
    smooth, other = probs[2], probs[5]
    assert smooth.X.shape == (576, 2) and other.X.shape == (828, 2)
    e = band(smooth, SPLIT_EPS)
    assert np.median(e) > 1e-4 and e.max() < 1e-3
    assert band(other, SPLIT_EPS).max() < 1e-5
    e_half = band(smooth, SPLIT_EPS / 2)
    assert 0.4 < np.median(e_half) / np.median(e) < 0.6
