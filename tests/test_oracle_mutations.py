"""Planted mistakes in the oracle (CPU only): each must be caught by one of the pins.

A pin that cannot tell a dropped term, a wrong sign or a transposed operand from the
right answer does not pin anything; these tests plant such mistakes with monkeypatch."""
import numpy as np
import pytest

import oracle as O
from oracle import sgks_oracle as OS
from workloads import small_problem


def _adjoint_gap(P):
    Aop, Lop = O.make_operators(P)
    rng = np.random.default_rng(0)
    gaps = []
    for op in (Aop, Lop):
        x, y = rng.standard_normal(op.shape[1]), rng.standard_normal(op.shape[0])
        gaps.append(abs(op.apply(x) @ y - x @ op.adjoint(y)) / (np.linalg.norm(x) * np.linalg.norm(y)))
    return max(gaps)


def test_sign_error_in_difference_adjoint_is_caught(monkeypatch):
    P = small_problem("deblur2d")
    assert _adjoint_gap(P) < 1e-13
    orig = OS._fd_axis_adj
    monkeypatch.setattr(OS, "_fd_axis_adj", lambda d, axis, n: -orig(d, axis, n))
    assert _adjoint_gap(P) > 1e-3


def test_dropped_regulariser_term_is_caught(monkeypatch):
    """Gradient without lam L^T L x: the basis is then K(A^T A, A^T b) only, and the
    full-basis pin (Tikhonov solution once d = n) no longer holds."""
    P = small_problem("deconv1d", n=14, s=30, lam=1e-1)
    Aop, Lop = O.make_operators(P)
    xd = O.direct_solve(Aop, Lop, P.b, P.lam)
    ok = O.sgks(P, iters=P.n - 3, sketched=False)["x"]
    monkeypatch.setattr(OS, "gradient", lambda A, L, b, lam, x: A.adjoint(A.apply(x) - b))
    bad = O.sgks(P, iters=P.n - 3, sketched=False)["x"]
    assert np.linalg.norm(ok - xd) / np.linalg.norm(xd) < 1e-8
    assert np.linalg.norm(bad - xd) / np.linalg.norm(xd) > 1e-6


def test_single_pass_loses_orthogonality_on_ill_conditioned_columns():
    rng = np.random.default_rng(4)
    # nearly dependent columns, like the late columns of the non-orthogonal sGKS basis
    M = rng.standard_normal((60, 1)) @ np.ones((1, 25)) + 1e-7 * rng.standard_normal((60, 25))
    res = {}
    for passes in (1, 2):
        Q, R = np.zeros((60, 0)), np.zeros((0, 0))
        for j in range(25):
            Q, R, _, _ = O.qr_append(Q, R, M[:, j], passes=passes)
        res[passes] = np.abs(Q.T @ Q - np.eye(25)).max()
    assert res[2] < 1e-13 < res[1]


def test_transposed_stacked_factor_is_caught(monkeypatch):
    rng = np.random.default_rng(5)
    d = 7
    RA, RL = np.triu(rng.standard_normal((d, d))), np.triu(rng.standard_normal((d, d)))
    dA = rng.standard_normal(d)
    orig = OS.projected_solve
    monkeypatch.setattr(OS, "projected_solve", lambda RA, RL, dA, lam: orig(RA, RL.T, dA, lam))
    y, _ = OS.projected_solve(RA, RL, dA, 0.3)
    grad = RA.T @ (RA @ y - dA) + 0.3 * RL.T @ (RL @ y)
    assert np.linalg.norm(grad) > 1e-6
