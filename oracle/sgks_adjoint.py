"""Plain FP64 CPU oracle for the derivative of sGKS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this module.  It differentiates the map (b, lambda) -> x_K of Algorithm 2 run for K
iterations, with or without the q = 0 refinement steps of the projected problem (Sec. 3.1),
for a loss l(x_K) whose gradient xbar = dl/dx_K is given, by a reverse sweep over the
iterations written from the algorithm's own equations:

  * x_j = W_j y_j, with y_j the minimiser of eq. (projected_sketched_bis).  In exact arithmetic
    y_j = G_j^{-1} h_j with G_j = U_j^T U_j + lambda V_j^T V_j, h_j = U_j^T c, U_j = S_A A W_j,
    V_j = S_L L W_j and c = S_A b (the normal equations of the sketched projected problem; the
    QR factors of eq. (updqr) are one way of solving them).  Its adjoint, for ybar given:
        z = G_j^{-1} ybar,   cbar += U_j z,   lambdabar -= (V_j z) . (V_j y_j),
        Wbar_j += P z^T + Q y^T,  P = A^T S_A^T (c - U_j y_j) - lambda L^T S_L^T V_j y_j,
                                  Q = -(A^T S_A^T U_j z + lambda L^T S_L^T V_j z).
  * x_j = W_j y_j itself gives ybar = W_j^T xbar_j and Wbar_j += xbar_j y_j^T.
  * With refinement, y_j = y^R is reached from y^0 (the projected solve above) by steps
    y^r = y^{r-1} - G_j^{-1} W_j^T rho(W_j y^{r-1}), rho(x) = H x - A^T b, H = A^T A + lambda L^T L
    (the gradient of eq. gradient).  The adjoint of one step, for ybar = ybar^r, with
    w = G_j^{-1} ybar and delta = y^{r-1} - y^r:
        ybar^{r-1} = ybar - W_j^T H W_j w,    bbar += A W_j w,
        lambdabar += (V_j w).(V_j delta) - (W_j w).(L^T L W_j y^{r-1}),
        Wbar_j += -rho(W_j y^{r-1}) w^T - (H W_j w) (y^{r-1})^T
                  + (A^T S_A^T U_j delta + lambda L^T S_L^T V_j delta) w^T
                  + (A^T S_A^T U_j w + lambda L^T S_L^T V_j w) delta^T,
    the last line from G_j = U_j^T U_j + lambda V_j^T V_j depending on W_j and lambda.  The
    projected solve's adjoint then runs with ybar^0 and y^0.
  * The new column r_j = A^T (A x_{j-1} - b) + lambda L^T L x_{j-1} (eq. gradient) gives, once
    its adjoint rbar = Wbar[:, d_j - 1] is complete (no later step touches it),
    xbar_{j-1} += (A^T A + lambda L^T L) rbar, bbar -= A rbar, lambdabar += rbar . L^T L x_{j-1}.
  * W_0 is an orthonormal basis of K_l(A^T A, A^T b) (Sec. 2.1).  Every x_j depends on W_0 only
    through its range, so W_0 may be written as K R_0^{-1} with K = [v, M v, ..., M^{l-1} v],
    v = A^T b, M = A^T A and R_0 = W_0^T K held fixed: Kbar = Wbar_0 R_0^{-T},
    vbar = sum_i M^i Kbar[:, i], bbar += A vbar.
  * Finally bbar += S_A^T cbar.

Pinned (tests/test_oracle_adjoint.py) by: central finite differences of the oracle's own
forward map (step 1e-6, FP64) for lambda and for random directions of b; and, once the basis
spans R^n, by the closed-form derivative of the sketched Tikhonov solution
x = (A^T S_A^T S_A A + lambda L^T S_L^T S_L L)^{-1} A^T S_A^T S_A b, which the sweep must
reproduce although it runs through every earlier step.
"""
from __future__ import annotations

import numpy as np

from .sgks_oracle import dense_matrix, make_operators, sgks, sketch_operator


def sgks_vjp(problem, iters, xbar, fwd=None, n_refine=0):
    """Reverse sweep: (bbar, lambdabar) = xbar^T d x_K / d(b, lambda) for K = iters.

    fwd: the oracle forward run with record_x=True (recomputed with n_refine refinement steps
    if None; otherwise its own refinement count is used).  Returns a dict with bbar (m),
    lambdabar, and the forward's x_K.
    """
    P = problem
    if P.sketch.kind not in ("sparse_sign", "gaussian", "srtt"):
        raise ValueError(P.sketch.kind)
    if fwd is None:
        fwd = sgks(P, iters=iters, n_refine=n_refine, record_x=True)
    Aop, Lop = make_operators(P)
    lam = float(P.lam)
    b = np.asarray(P.b, dtype=np.float64)
    SA = sketch_operator(P.sketch, 0, P.m)
    SL = sketch_operator(P.sketch, 1, P.p)
    c = SA @ b
    W = fwd["W"]
    ys, xs, yrs = fwd["ys"], fwd["xs"], fwd["yrs"]
    K = len(ys) - 1
    ell = W.shape[1] - K
    # U = S_A A W, V = S_L L W, column by column (the sketched columns of eq. updqr)
    U = np.stack([SA @ Aop.apply(W[:, i]) for i in range(W.shape[1])], axis=1)
    V = np.stack([SL @ Lop.apply(W[:, i]) for i in range(W.shape[1])], axis=1)

    def AtSAt(v):
        return Aop.adjoint(SA.T @ v)

    def LtSLt(v):
        return Lop.adjoint(SL.T @ v)

    def H(v):   # A^T A + lambda L^T L
        return Aop.adjoint(Aop.apply(v)) + lam * Lop.adjoint(Lop.apply(v))

    def LtL(v):
        return Lop.adjoint(Lop.apply(v))

    Wbar = np.zeros_like(W)
    bbar = np.zeros(P.m)
    cbar = np.zeros(len(c))
    lbar = 0.0
    xbar_j = np.array(xbar, dtype=np.float64)
    for j in range(K, -1, -1):
        d = ell + j
        Wj, Uj, Vj = W[:, :d], U[:, :d], V[:, :d]
        chain = yrs[j]
        ybar = Wj.T @ xbar_j
        Wbar[:, :d] += np.outer(xbar_j, chain[-1])
        G = Uj.T @ Uj + lam * (Vj.T @ Vj)
        for r in range(len(chain) - 1, 0, -1):   # refinement steps, last first
            yprev = chain[r - 1]
            delta = yprev - chain[r]
            w = np.linalg.solve(G, ybar)
            Ww = Wj @ w
            AWw = Aop.apply(Ww)
            HWw = Aop.adjoint(AWw) + lam * LtL(Ww)
            xprev = Wj @ yprev
            rho = Aop.adjoint(Aop.apply(xprev) - b) + lam * LtL(xprev)
            bbar += AWw
            lg, Wg = _preconditioner_terms(Uj, Vj, lam, w, delta, AtSAt, LtSLt)
            lbar += lg - float(Ww @ LtL(xprev))
            Wbar[:, :d] += Wg - np.outer(rho, w) - np.outer(HWw, yprev)
            ybar = ybar - Wj.T @ HWw
        y = chain[0]
        z = np.linalg.solve(G, ybar)
        Uy, Uz, Vy, Vz = Uj @ y, Uj @ z, Vj @ y, Vj @ z
        cbar += Uz
        lbar -= float(Vz @ Vy)
        Pv = AtSAt(c - Uy) - lam * LtSLt(Vy)
        Qv = -(AtSAt(Uz) + lam * LtSLt(Vz))
        Wbar[:, :d] += np.outer(Pv, z) + np.outer(Qv, y)
        if j == 0:
            break
        rbar = Wbar[:, d - 1]
        x_prev = xs[j - 1]
        xbar_j = H(rbar)
        bbar -= Aop.apply(rbar)
        lbar += float(rbar @ Lop.adjoint(Lop.apply(x_prev)))
    # W_0 = K R_0^{-1} with R_0 fixed: the Krylov vectors v, M v, ... of v = A^T b
    W0 = W[:, :ell]
    v = Aop.adjoint(b)
    Kry = [v]
    for _ in range(1, ell):
        Kry.append(Aop.adjoint(Aop.apply(Kry[-1])))
    Kry = np.stack(Kry, axis=1)
    R0 = W0.T @ Kry
    Kbar = Wbar[:, :ell] @ np.linalg.inv(R0).T
    vbar = np.zeros(P.n)
    for i in range(ell - 1, -1, -1):   # Horner: vbar = sum_i M^i Kbar[:, i]
        vbar = Kbar[:, i] + (Aop.adjoint(Aop.apply(vbar)) if i < ell - 1 else 0.0)
    bbar += Aop.apply(vbar)
    bbar += SA.T @ cbar
    return dict(bbar=bbar, lambdabar=lbar, x=xs[-1], fwd=fwd)


def _preconditioner_terms(Uj, Vj, lam, w, delta, AtSAt, LtSLt):
    """The contribution of G_j = U_j^T U_j + lambda V_j^T V_j (through W_j and lambda) to the
    adjoint of one refinement step: lambdabar += (V w).(V delta), and Wbar gains
    (A^T S_A^T U delta + lambda L^T S_L^T V delta) w^T + (A^T S_A^T U w + lambda L^T S_L^T V w) delta^T."""
    a1 = AtSAt(Uj @ delta) + lam * LtSLt(Vj @ delta)
    a2 = AtSAt(Uj @ w) + lam * LtSLt(Vj @ w)
    return float((Vj @ w) @ (Vj @ delta)), np.outer(a1, w) + np.outer(a2, delta)


def loss_and_grad(problem, iters, target=None, n_refine=0):
    """l = ||x_K - target||^2 (target = x_true by default) and its gradient w.r.t. (b, lambda),
    for the solve with n_refine refinement steps per iteration."""
    P = problem
    t = np.asarray(P.x_true if target is None else target, dtype=np.float64)
    fwd = sgks(P, iters=iters, n_refine=n_refine, record_x=True)
    x = fwd["xs"][-1]
    g = sgks_vjp(P, iters, 2.0 * (x - t), fwd=fwd)
    return float(np.sum((x - t) ** 2)), g["bbar"], g["lambdabar"]


def sketched_tikhonov_vjp(problem, xbar):
    """Closed-form pin: x = (A^T S_A^T S_A A + lam L^T S_L^T S_L L)^{-1} A^T S_A^T S_A b (dense, tiny n);
    returns (x, bbar, lambdabar) for the given xbar."""
    P = problem
    Aop, Lop = make_operators(P)
    A = dense_matrix(Aop, P.n)
    L = dense_matrix(Lop, P.n)
    SA = sketch_operator(P.sketch, 0, P.m)
    SL = sketch_operator(P.sketch, 1, P.p)
    SA = SA.toarray() if hasattr(SA, "toarray") else SA
    SL = SL.toarray() if hasattr(SL, "toarray") else SL
    lam = float(P.lam)
    SAA, SLL = SA @ A, SL @ L
    M = SAA.T @ SAA + lam * (SLL.T @ SLL)
    b = np.asarray(P.b, dtype=np.float64)
    x = np.linalg.solve(M, SAA.T @ (SA @ b))
    w = np.linalg.solve(M, np.asarray(xbar, dtype=np.float64))   # M symmetric
    bbar = SA.T @ (SAA @ w)
    lbar = -float(w @ (SLL.T @ (SLL @ x)))
    return x, bbar, lbar
