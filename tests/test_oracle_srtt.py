"""Pins of the oracle's SRTT sketch (eq. sketching_trig): S = sqrt(h/s) D F E with F the
orthonormal DCT-II, E a Rademacher diagonal and D s sampled rows of the identity."""
import numpy as np

import oracle as O
from oracle.sgks_oracle import SRTT, sketch_operator
from workloads import small_problem
from workloads.configs import srtt_sketch


def test_full_sampling_is_orthogonal():
    h = 40
    signs = np.where(np.random.default_rng(0).random(h) < 0.5, -1.0, 1.0)
    M = SRTT(signs, np.arange(h)).toarray()          # s = h: sqrt(1) F E
    assert np.abs(M.T @ M - np.eye(h)).max() < 1e-13


def test_dct_basis_vector_maps_to_one_row():
    """x_i = cos(pi k0 (2i+1) / (2h)) is f_{k0} / c_{k0} for the DCT-II basis vector f_{k0}, so
    F x = sqrt(h/2) e_{k0} (k0 > 0): S x is sqrt(h/s) sqrt(h/2) in the row that samples k0."""
    h, k0 = 50, 7
    i = np.arange(h)
    x = np.cos(np.pi * k0 * (2 * i + 1) / (2 * h))
    rows = np.array([3, 7, 20, 41])
    y = SRTT(np.ones(h), rows) @ x
    want = np.zeros(len(rows))
    want[1] = np.sqrt(h / len(rows)) * np.sqrt(h / 2)
    assert np.abs(y - want).max() < 1e-12 * np.abs(want).max()


def test_transpose_is_the_adjoint():
    d = srtt_sketch(12, 64, 70, seed=3)
    rng = np.random.default_rng(1)
    for stream, h in ((0, 64), (1, 70)):
        S = sketch_operator(d, stream, h)
        v, u = rng.standard_normal(h), rng.standard_normal(12)
        assert abs((S @ v) @ u - v @ (S.T @ u)) < 1e-12 * np.linalg.norm(v) * np.linalg.norm(u) * 10


def test_expected_gram_is_identity():
    """E[S^T S] = I over the random signs and row samples (Monte Carlo, h = 24, s = 6)."""
    h, s, trials = 24, 6, 4000
    rng = np.random.default_rng(7)
    acc = np.zeros((h, h))
    for _ in range(trials):
        signs = rng.choice([-1.0, 1.0], size=h)
        rows = rng.choice(h, size=s, replace=False)
        M = SRTT(signs, rows).toarray()
        acc += M.T @ M
    acc /= trials
    assert np.abs(np.diag(acc) - 1.0).max() < 0.08
    assert np.abs(acc - np.diag(np.diag(acc))).max() < 0.08


def test_sgks_with_srtt_reaches_the_sketched_tikhonov_solution():
    """Once the basis spans R^n, sGKS with the SRTT sketch equals the dense solution of the
    sketched functional (as for the other sketches)."""
    P = small_problem("ct2d", N=4, nbins=7, iters=13, s=20)      # n = 16 = ell + 13, m = 168, p = 24
    P.sketch = srtt_sketch(20, P.m, P.p, seed=2)
    out = O.sgks(P, iters=13, n_refine=0)
    assert out["breakdowns"] == 0
    Aop, Lop = O.make_operators(P)
    SA = sketch_operator(P.sketch, 0, P.m)
    SL = sketch_operator(P.sketch, 1, P.p)
    x = O.direct_solve(Aop, Lop, np.asarray(P.b, dtype=np.float64), P.lam, SA.toarray(), SL.toarray())
    assert np.linalg.norm(out["x"] - x) <= 1e-9 * np.linalg.norm(x)
