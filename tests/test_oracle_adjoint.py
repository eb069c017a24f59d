"""Pins of the oracle's reverse sweep (oracle/sgks_adjoint.py).

The derivative of x_K(b, lambda) is checked against (1) central finite differences of the
oracle's own forward map in FP64 with step 1e-6, for lambda and random directions of b, on CSR,
convolution and CT operators; and (2) the closed-form derivative of the sketched Tikhonov
solution once the basis spans R^n, which the sweep has to reproduce through every earlier step.
"""
import numpy as np
import pytest

import oracle as O
from oracle.sgks_adjoint import loss_and_grad, sgks_vjp, sketched_tikhonov_vjp
from workloads import small_problem
from workloads.problem import SketchDesc


def _fd(P, it, h=1e-6, seed=3, ndir=2, n_refine=0):
    L0, bb, lb = loss_and_grad(P, it, n_refine=n_refine)
    lam0 = P.lam
    P.lam = lam0 + h
    lp = loss_and_grad(P, it, n_refine=n_refine)[0]
    P.lam = lam0 - h
    lm = loss_and_grad(P, it, n_refine=n_refine)[0]
    P.lam = lam0
    out = [(lb, (lp - lm) / (2 * h))]
    rng = np.random.default_rng(seed)
    b0 = np.array(P.b, dtype=np.float64)
    for _ in range(ndir):
        dv = rng.standard_normal(P.m)
        P.b = b0 + h * dv
        lp = loss_and_grad(P, it, n_refine=n_refine)[0]
        P.b = b0 - h * dv
        lm = loss_and_grad(P, it, n_refine=n_refine)[0]
        P.b = b0
        out.append((float(bb @ dv), (lp - lm) / (2 * h)))
    return out


@pytest.mark.parametrize("kind,iters", [("seismic2d", 12), ("deblur2d", 10), ("ct2d", 10), ("deconv1d", 8)])
def test_adjoint_matches_central_differences(kind, iters):
    P = small_problem(kind, iters=iters)
    P.n_refine = 0
    for an, fd in _fd(P, iters):
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-9, (kind, an, fd)


@pytest.mark.parametrize("kind,iters,n_refine", [("seismic2d", 10, 1), ("deblur2d", 8, 2), ("ct2d", 8, 2),
                                                  ("deconv1d", 8, 3)])
def test_adjoint_with_refinement_matches_central_differences(kind, iters, n_refine):
    """The sweep through the q = 0 refinement steps (their dependence on y, W, b and lambda,
    including lambda and W inside the sketched preconditioner G) against central differences
    of the refined forward map."""
    P = small_problem(kind, iters=iters)
    for an, fd in _fd(P, iters, n_refine=n_refine):
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-9, (kind, n_refine, an, fd)


@pytest.mark.parametrize("n_refine", [0, 2])
def test_adjoint_with_srtt_sketch_matches_central_differences(n_refine):
    """The sweep with the subsampled randomized trigonometric transform (eq. sketching_trig) as
    S_A and S_L, without and with refinement steps, against central differences."""
    from workloads.configs import srtt_sketch
    P = small_problem("ct2d", iters=8)
    P.sketch = srtt_sketch(40, P.m, P.p, seed=2)
    for an, fd in _fd(P, 8, n_refine=n_refine):
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-9, (n_refine, an, fd)


def test_refinement_adjoint_terms_are_all_needed(monkeypatch):
    """A planted mistake: dropping the preconditioner's dependence on W and lambda (the G_j terms
    of the refinement adjoint) must fail the finite-difference pin, so the pin is not blind to
    those terms."""
    import oracle.sgks_adjoint as OA
    P = small_problem("seismic2d", iters=6)
    def no_g_terms(Uj, Vj, lam, w, delta, AtSAt, LtSLt):
        return 0.0, np.zeros((AtSAt(Uj @ w).shape[0], len(w)))

    monkeypatch.setattr(OA, "_preconditioner_terms", no_g_terms)
    errs = [abs(an - fd) / abs(fd) for an, fd in _fd(P, 6, n_refine=2)]
    assert max(errs) > 1e-4, errs


def test_adjoint_equals_closed_form_once_basis_spans_space():
    """n = 8, ell + K = 8: x_K is the sketched Tikhonov solution, so its derivative is known in
    closed form; the sweep reaches it although every step's basis depends on b and lambda."""
    P = small_problem("deconv1d", n=8, s=40, iters=5, lam=1e-1)
    P.sketch = SketchDesc("sparse_sign", 40, 8, 0)
    fwd = O.sgks(P, iters=5, n_refine=0, record_x=True)
    assert fwd["breakdowns"] == 0
    xbar = np.random.default_rng(0).standard_normal(P.n)
    xc, bb_c, lb_c = sketched_tikhonov_vjp(P, xbar)
    assert np.linalg.norm(fwd["xs"][-1] - xc) <= 1e-12 * np.linalg.norm(xc)
    g = sgks_vjp(P, 5, xbar, fwd=fwd)
    assert np.linalg.norm(g["bbar"] - bb_c) <= 1e-9 * np.linalg.norm(bb_c)
    assert abs(g["lambdabar"] - lb_c) <= 1e-9 * abs(lb_c)


def test_adjoint_is_linear_in_xbar():
    P = small_problem("seismic2d", iters=6)
    fwd = O.sgks(P, iters=6, n_refine=0, record_x=True)
    rng = np.random.default_rng(1)
    a, c = rng.standard_normal(P.n), rng.standard_normal(P.n)
    ga, gc = sgks_vjp(P, 6, a, fwd=fwd), sgks_vjp(P, 6, c, fwd=fwd)
    g = sgks_vjp(P, 6, 2.0 * a - 3.0 * c, fwd=fwd)
    ref = 2.0 * ga["bbar"] - 3.0 * gc["bbar"]
    assert np.linalg.norm(g["bbar"] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert abs(g["lambdabar"] - (2.0 * ga["lambdabar"] - 3.0 * gc["lambdabar"])) <= 1e-12 * abs(g["lambdabar"]) + 1e-15


def test_planted_adjoint_mistake_is_caught(monkeypatch):
    """A wrong L^T (1 % off) breaks the exactness the sweep relies on: the FD pin must fail."""
    import oracle.sgks_adjoint as OA
    import oracle.sgks_oracle as OS
    real = OS.make_operators

    def skewed(problem):
        Aop, Lop = real(problem)
        adj = Lop.adjoint
        Lop.adjoint = lambda v: 1.01 * adj(v)
        return Aop, Lop

    monkeypatch.setattr(OS, "make_operators", skewed)
    monkeypatch.setattr(OA, "make_operators", skewed)
    P = small_problem("seismic2d", iters=8)
    P.n_refine = 0
    worst = max(abs(an - fd) / abs(fd) for an, fd in _fd(P, 8))
    assert worst > 1e-4
