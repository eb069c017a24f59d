"""Pins of the FP64 oracle against facts fixed outside it (paper statements, closed forms,
published test vectors, library routines, brute force on tiny inputs).  CPU only."""
import os

import numpy as np
import pytest
import scipy.signal
import scipy.sparse as sp

import oracle as O
from oracle import sgks_oracle as OS
from workloads import small_problem
from workloads.problem import RegDesc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


# ------------------------------------------------------------------------------ sketch

def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        want = [int(l) for l in f if l.strip() and not l.startswith("#")]
    assert OS.splitmix64_sequence(1234567, len(want)) == want


@pytest.mark.parametrize("s,zeta", [(40, 8), (400, 8), (9, 9), (16, 1)])
def test_sparse_sign_structure(s, zeta):
    h = 3000
    rows, signs = O.sparse_sign_rows(7, 0, h, s, zeta)
    assert rows.min() >= 0 and rows.max() < s
    srt = np.sort(rows, axis=1)
    assert (np.diff(srt, axis=1) > 0).all(), "rows of one column must be distinct"
    assert set(np.unique(signs)) <= {-1.0, 1.0}
    # each column of S has unit norm: diag(S^T S) = 1 exactly
    S = O.sketch_operator(type("D", (), dict(kind="sparse_sign", s=s, zeta=zeta, seed=7))(), 0, h)
    assert np.allclose(np.asarray(S.multiply(S).sum(axis=0)).ravel(), 1.0, atol=1e-15)


def test_sparse_sign_uniform_and_unbiased():
    s, zeta, h = 50, 4, 40000
    rows, signs = O.sparse_sign_rows(3, 1, h, s, zeta)
    counts = np.bincount(rows.ravel(), minlength=s)
    exp = h * zeta / s
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 100.0, chi2                       # 49 dof: mean 49, sd ~10
    assert abs(signs.mean()) < 4.0 / np.sqrt(signs.size)


def test_sparse_sign_streams_differ():
    a, _ = O.sparse_sign_rows(0, 0, 500, 64, 8)
    b, _ = O.sparse_sign_rows(0, 1, 500, 64, 8)
    c, _ = O.sparse_sign_rows(1, 0, 500, 64, 8)
    assert (a != b).any() and (a != c).any()


def test_sketch_expectation_identity():
    """E[S^T S] = I (the scaling of Sec. 2.2), Monte Carlo over seeds."""
    h, s, zeta, T = 12, 20, 3, 4000
    acc = np.zeros((h, h))
    for seed in range(T):
        rows, signs = O.sparse_sign_rows(seed, 0, h, s, zeta)
        S = np.zeros((s, h))
        S[rows, np.arange(h)[:, None]] = signs / np.sqrt(zeta)
        acc += S.T @ S
    acc /= T
    assert np.abs(acc - np.eye(h)).max() < 0.05


def test_sketch_is_subspace_embedding():
    """Def. 1: singular values of S Q (Q orthonormal, q-dim) close to 1 for s >> q."""
    h, q = 5000, 10
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((h, q)))
    D = type("D", (), dict(kind="sparse_sign", s=400, zeta=8, seed=5))()
    sv = np.linalg.svd(O.sketch_operator(D, 0, h) @ Q, compute_uv=False)
    eps = max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)
    assert eps < 0.5, eps


# --------------------------------------------------------------------------- operators

def _D(n):
    return np.eye(n)[1:] - np.eye(n)[:-1]


def test_grad2d_matches_kronecker_definition():
    nx, ny = 7, 5
    P = small_problem("deblur2d", nx=nx, ny=ny)
    _, Lop = O.make_operators(P)
    Lk = np.vstack([np.kron(np.eye(ny), _D(nx)), np.kron(_D(ny), np.eye(nx))])  # eq. reg_matrix
    assert np.allclose(OS.dense_matrix(Lop, nx * ny), Lk, atol=0, rtol=0)


def test_spacetime_matches_kronecker_definition():
    nx, ny, nt = 5, 4, 3
    Lop = OS._reg(RegDesc("spacetime", nx=nx, ny=ny, nt=nt))
    Ix, Iy, It = np.eye(nx), np.eye(ny), np.eye(nt)
    Psi = np.vstack([np.kron(It, np.kron(Iy, _D(nx))),       # eq. spacetime_tik
                     np.kron(It, np.kron(_D(ny), Ix)),
                     np.kron(_D(nt), np.kron(Iy, Ix))])
    assert Psi.shape[0] == RegDesc("spacetime", nx=nx, ny=ny, nt=nt).p
    assert np.array_equal(OS.dense_matrix(Lop, nx * ny * nt), Psi)


def test_fd1_and_laplace_match_definition():
    Lop = OS._reg(RegDesc("fd1", nx=9))
    assert np.array_equal(OS.dense_matrix(Lop, 9), _D(9))
    nx, ny = 6, 4
    Lap = OS.dense_matrix(OS._reg(RegDesc("laplace2d", nx=nx, ny=ny)), nx * ny)
    T1 = lambda k: 2 * np.eye(k) - np.eye(k, k=1) - np.eye(k, k=-1)  # noqa: E731
    assert np.array_equal(Lap, np.kron(np.eye(ny), T1(nx)) + np.kron(T1(ny), np.eye(nx)))


def test_conv2d_matches_scipy_convolve2d():
    P = small_problem("deblur2d", nx=13, ny=9)
    Aop, _ = O.make_operators(P)
    x = np.random.default_rng(1).standard_normal(13 * 9)
    ref = scipy.signal.convolve2d(x.reshape(9, 13), P.A.psf.astype(np.float64), mode="same")
    assert rel(Aop.apply(x), ref.ravel()) < 1e-15
    # a non-symmetric PSF catches a flipped kernel
    P.A.psf = np.random.default_rng(2).random((5, 3)).astype(np.float32)
    Aop, _ = O.make_operators(P)
    ref = scipy.signal.convolve2d(x.reshape(9, 13), P.A.psf.astype(np.float64), mode="same")
    assert rel(Aop.apply(x), ref.ravel()) < 1e-15


@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_adjoint_identity(kind):
    P = small_problem(kind)
    Aop, Lop = O.make_operators(P)
    rng = np.random.default_rng(3)
    for op in (Aop, Lop):
        x = rng.standard_normal(op.shape[1])
        y = rng.standard_normal(op.shape[0])
        lhs, rhs = op.apply(x) @ y, x @ op.adjoint(y)
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))


# ------------------------------------------------------------------------ building blocks

def test_initial_basis_spans_krylov_space():
    P = small_problem("deblur2d")
    Aop, _ = O.make_operators(P)
    V = O.initial_basis(Aop, P.b, 3)
    assert np.abs(V.T @ V - np.eye(3)).max() < 1e-14
    k = Aop.adjoint(P.b)
    for _ in range(3):
        assert np.linalg.norm(k - V @ (V.T @ k)) < 1e-10 * np.linalg.norm(k)
        k = Aop.adjoint(Aop.apply(k))


def test_qr_append_reproduces_matrix():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((60, 25)) @ np.diag(np.logspace(0, -8, 25))
    Q, R = np.zeros((60, 0)), np.zeros((0, 0))
    for j in range(25):
        Q, R, _, _ = O.qr_append(Q, R, M[:, j], passes=2)
    assert np.linalg.norm(Q @ R - M) <= 1e-13 * np.linalg.norm(M)
    assert np.abs(Q.T @ Q - np.eye(25)).max() < 1e-13
    assert np.allclose(R, np.triu(R))


def test_qr_append_breakdown():
    Q, R = np.zeros((10, 0)), np.zeros((0, 0))
    u = np.arange(10.0)
    Q, R, _, b1 = O.qr_append(Q, R, u)
    Q, R, rho, b2 = O.qr_append(Q, R, 3 * u)
    assert not b1 and b2 and rho == 0.0 and not Q[:, 1].any()


def test_projected_solve_satisfies_normal_equations():
    rng = np.random.default_rng(5)
    d = 9
    RA, RL = np.triu(rng.standard_normal((d, d))), np.triu(rng.standard_normal((d, d)))
    dA, lam = rng.standard_normal(d), 0.3
    y, T = O.projected_solve(RA, RL, dA, lam)
    grad = RA.T @ (RA @ y - dA) + lam * RL.T @ (RL @ y)
    assert np.linalg.norm(grad) < 1e-12 * np.linalg.norm(RA.T @ dA)
    assert np.allclose(T.T @ T, RA.T @ RA + lam * RL.T @ RL, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------- whole solver

@pytest.mark.parametrize("kind", ["deconv1d", "dynct"])
def test_full_basis_reaches_direct_solve(kind):
    """Once the basis spans R^n, GKS and sGKS_0 return the Tikhonov solution."""
    if kind == "deconv1d":
        P = small_problem("deconv1d", n=14, s=30, lam=1e-1)
    else:
        P = small_problem("dynct", N=4, frames=2, s=60, lam=0.5, n_refine=0)
    n = P.n
    Aop, Lop = O.make_operators(P)
    xd = O.direct_solve(Aop, Lop, P.b, P.lam)
    assert rel(O.gks(P, iters=n - 3)["x"], xd) < 1e-10
    assert rel(O.sgks(P, iters=n - 3, sketched=False)["x"], xd) < 1e-8


def test_full_basis_reaches_sketched_direct_solve():
    """sGKS with d = n solves the sketched functional of eq. (tik_new_sketched) exactly."""
    P = small_problem("deconv1d", n=14, s=30, lam=1e-1)
    Aop, Lop = O.make_operators(P)
    SA, SL = O.sketch_operator(P.sketch, 0, P.m), O.sketch_operator(P.sketch, 1, P.p)
    xs = O.direct_solve(Aop, Lop, P.b, P.lam, SA, SL)
    assert rel(O.sgks(P, iters=P.n - 3)["x"], xs) < 1e-9


def test_proposition1_gks_equals_sgks0():
    """Proposition 1: with range W_0 = range V_0, sGKS_0 iterates equal GKS iterates."""
    P = small_problem("deblur2d", precision="fp64", n_refine=0)
    g = O.gks(P, iters=10, record_x=True)
    s0 = O.sgks(P, iters=10, sketched=False, record_x=True)
    for k, (a, b) in enumerate(zip(g["xs"], s0["xs"])):
        assert rel(b, a) < 1e-9, (k, rel(b, a))


def test_proposition2_quasi_optimality():
    """Proposition 2: J(W y_sGKS) <= (1+gamma)/(1-theta) J(W y_sGKS0) with measured eps."""
    P = small_problem("ct2d", s=60, iters=8)
    out = O.sgks(P, record_state=True)
    Aop, Lop = O.make_operators(P)
    W = out["W"]
    AW = np.stack([Aop.apply(w) for w in W.T], 1)
    LW = np.stack([Lop.apply(w) for w in W.T], 1)
    SA, SL = O.sketch_operator(P.sketch, 0, P.m), O.sketch_operator(P.sketch, 1, P.p)

    def eps(S, M):
        Q, _ = np.linalg.qr(M)
        sv = np.linalg.svd(S @ Q, compute_uv=False)
        return max(sv.max() ** 2 - 1, 1 - sv.min() ** 2)

    eA, eL = eps(SA, np.column_stack([AW, P.b])), eps(SL, LW)
    th, ga = min(eA, eL), max(eA, eL)
    assert th < 1
    M0 = np.vstack([AW, np.sqrt(P.lam) * LW])
    y0 = np.linalg.lstsq(M0, np.concatenate([P.b, np.zeros(P.p)]), rcond=None)[0]
    J = lambda y: O.tikhonov_functional(Aop, Lop, P.b, P.lam, W @ y)  # noqa: E731
    assert J(out["y"]) <= (1 + ga) / (1 - th) * J(y0) * (1 + 1e-12)
    assert J(y0) <= J(out["y"]) * (1 + 1e-12)     # y0 is optimal over range(W)


def test_functional_nonincreasing():
    """Nested subspaces: the GKS functional and the sGKS sketched functional never increase."""
    P = small_problem("seismic2d", iters=12)
    Aop, Lop = O.make_operators(P)
    g = O.gks(P, record_x=True)
    J = [O.tikhonov_functional(Aop, Lop, P.b, P.lam, x) for x in g["xs"]]
    assert all(J[k + 1] <= J[k] * (1 + 1e-12) for k in range(len(J) - 1))
    SA, SL = O.sketch_operator(P.sketch, 0, P.m), O.sketch_operator(P.sketch, 1, P.p)
    s = O.sgks(P, record_x=True)
    Js = [np.sum((SA @ (Aop.apply(x) - P.b)) ** 2) + P.lam * np.sum((SL @ Lop.apply(x)) ** 2)
          for x in s["xs"]]
    assert all(Js[k + 1] <= Js[k] * (1 + 1e-10) for k in range(len(Js) - 1))


def test_gradient_orthogonal_to_basis():
    """V_k^T r_{k+1} = 0 for GKS and W_k^T r_{k+1} = 0 for sGKS_0 (normal equations, Sec. 2.1)."""
    P = small_problem("deblur2d", precision="fp64", n_refine=0)
    Aop, Lop = O.make_operators(P)
    s0 = O.sgks(P, iters=6, sketched=False)
    r = OS.gradient(Aop, Lop, P.b, P.lam, s0["x"])
    W = s0["W"]
    assert np.linalg.norm(W.T @ r) < 1e-9 * np.linalg.norm(W, 2) * np.linalg.norm(r)
    g = O.gks(P, iters=6)
    r = OS.gradient(Aop, Lop, P.b, P.lam, g["x"])
    assert np.linalg.norm(g["V"].T @ r) < 1e-9 * np.linalg.norm(r)


def test_refinement_converges_to_unsketched_solution():
    """The refinement's fixed point is y_sGKS0 over the same W (Sec. 3.1, Sec. 4.3)."""
    P = small_problem("deblur2d", precision="fp64", n_refine=0, s=300)
    out = O.sgks(P, iters=8, record_state=True)
    Aop, Lop = O.make_operators(P)
    W = out["W"]
    y, T = O.projected_solve(out["RA"], out["RL"], out["dA"], P.lam)
    AW = np.stack([Aop.apply(w) for w in W.T], 1)
    LW = np.stack([Lop.apply(w) for w in W.T], 1)
    y0 = np.linalg.lstsq(np.vstack([AW, np.sqrt(P.lam) * LW]),
                         np.concatenate([P.b, np.zeros(P.p)]), rcond=None)[0]
    errs = []
    for _ in range(30):
        errs.append(rel(W @ y, W @ y0))
        y = O.refine_step(Aop, Lop, P.b, P.lam, W, y, T)
    assert errs[-1] < 1e-11
    # the error contracts at the spectral radius of I - (T^T T)^{-1} H, H the unsketched Hessian
    M0 = np.vstack([AW, np.sqrt(P.lam) * LW])
    rho = max(abs(np.linalg.eigvals(np.eye(len(y)) - np.linalg.solve(T.T @ T, M0.T @ M0))))
    assert rho < 1
    assert errs[15] <= errs[0] * (rho + 0.05) ** 15
