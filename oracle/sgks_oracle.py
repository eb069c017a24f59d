"""Plain FP64 CPU oracle for GKS and sGKS -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
leg may import this module.  It is written from the paper (Palitta & Pasha, "A Sketched
Generalized Krylov Subspace Method for Large-Scale Regularization"), step by step in the
paper's order and notation, with NumPy / SciPy primitives (matmul, sparse matvec, QR,
triangular solve) as the only library steps.  Everything is float64.

What each function follows, and what pins it (tests/test_oracle_*.py):
  splitmix64_mix       SplitMix64 finalizer (Steele, Lea, Flood 2014; Vigna's splitmix64.c).
                       Pinned by the published output sequence for seed 1234567.
  sparse_sign_rows     sparse-sign sketch positions/signs (not in the paper; the paper allows
                       any oblivious embedding, Sec. 2.2).  Pinned by properties: zeta distinct
                       rows per column in [0, s), E[S^T S] = I (Monte Carlo), row uniformity.
  make_operators       A and L of the workloads: dense, CSR, 2D convolution; fd1, grad2d
                       (eq. reg_matrix), 5-point Laplacian, space-time Psi (eq. spacetime_tik).
                       Pinned by Kronecker constructions of eq. reg_matrix / spacetime_tik,
                       scipy.signal.convolve2d, and the adjoint identity <Ax,y> = <x,A^T y>.
  initial_basis        orthonormal basis of K_l(A^T A, A^T b) (Sec. 2.1, Sec. 4: l = 3).
                       Pinned by orthonormality and by spanning the Krylov space.
  qr_append            rank-one column append of eq. (updqr) and the align block under it,
                       applied twice (CGS2) by default.  Pinned by QR = M and Q^T Q = I.
  projected_solve      eq. (projected_sketched_bis): Householder QR of [R_A; sqrt(lam) R_L],
                       rebuilt from scratch each call, then back substitution.
  combine              x = W y (a matmul).
  refine_step          one sketch-preconditioned refinement step of the projected problem,
                       the q = 0 setting of Sec. 4.3 (no inner iteration).  Pinned by
                       convergence to the unsketched projected solution (eq. sGKS_noSASL).
  sgks                 Algorithm 2 (sGKS), optionally with S = I (sGKS_0 of eq. sGKS_noSASL).
  gks                  Algorithm 1 (GKS) with the loss-ratio test of eq. (loss_criterion).
                       sgks/gks are pinned by: the dense direct solve once the basis spans
                       R^n; Proposition 1 (GKS == sGKS_0); Proposition 2 (quasi-optimality);
                       non-increasing functional over nested subspaces; V^T r = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg
import scipy.sparse as sp

U64 = np.uint64
_GOLDEN = 0x9E3779B97F4A7C15


# ----------------------------------------------------------------------------- sketch

def splitmix64_mix(z):
    """SplitMix64 output function (the 'mix64' finalizer) on uint64 values."""
    z = np.asarray(z, dtype=U64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
        z = z ^ (z >> U64(31))
    return z


def splitmix64_sequence(seed: int, count: int):
    """The SplitMix64 generator: state += golden gamma, output mix64(state)."""
    out = []
    state = int(seed) % 2 ** 64
    for _ in range(count):
        state = (state + _GOLDEN) % 2 ** 64
        out.append(int(splitmix64_mix(U64(state))))
    return out


def sparse_sign_rows(seed: int, stream: int, h: int, s: int, zeta: int, max_draws: int = 256):
    """Positions and signs of the sparse-sign sketch S (s x h), zeta nonzeros per column.

    Column j draws c = 0, 1, 2, ...: hv = mix64(mix64(2*seed + stream) XOR (j*256 + c)),
    row = floor((hv >> 32) * s / 2^32) (multiply-shift range reduction), sign = -1 if hv is
    odd else +1; a row already taken by column j is rejected and the next draw is used.
    Returns rows (h, zeta) int64 in draw order and signs (h, zeta) float64.
    """
    if not (1 <= zeta <= s):
        raise ValueError("need 1 <= zeta <= s")
    key = splitmix64_mix(U64((2 * int(seed) + int(stream)) % 2 ** 64))
    rows = np.full((h, zeta), -1, dtype=np.int64)
    signs = np.zeros((h, zeta), dtype=np.float64)
    count = np.zeros(h, dtype=np.int64)
    j = np.arange(h, dtype=U64)
    for c in range(max_draws):
        active = np.flatnonzero(count < zeta)
        if active.size == 0:
            break
        hv = splitmix64_mix(key ^ ((j[active] << U64(8)) | U64(c)))
        r = (((hv >> U64(32)) * U64(s)) >> U64(32)).astype(np.int64)
        sg = np.where((hv & U64(1)) == U64(1), -1.0, 1.0)
        dup = (rows[active] == r[:, None]).any(axis=1)
        acc = active[~dup]
        rows[acc, count[acc]] = r[~dup]
        signs[acc, count[acc]] = sg[~dup]
        count[acc] += 1
    if (count < zeta).any():
        raise RuntimeError("sparse-sign draw limit reached")
    return rows, signs


def sketch_operator(desc, stream: int, h: int):
    """S_A (stream 0, h = m) or S_L (stream 1, h = p) as a SciPy sparse or dense matrix.

    All sketches are scaled so that E[S^T S] = I (Sec. 2.2 scales the SRTT by sqrt(n/s)):
    Gaussian entries N(0, 1/s), sparse-sign values +-1/sqrt(zeta).
    """
    if desc.kind == "gaussian":
        M = desc.SA if stream == 0 else desc.SL
        assert M.shape == (desc.s, h)
        return np.asarray(M, dtype=np.float64)
    if desc.kind == "srtt":
        signs = desc.signs_A if stream == 0 else desc.signs_L
        rows = desc.rows_A if stream == 0 else desc.rows_L
        assert len(signs) == h and len(rows) == desc.s
        return SRTT(np.asarray(signs, dtype=np.float64), np.asarray(rows, dtype=np.int64))
    rows, signs = sparse_sign_rows(desc.seed, stream, h, desc.s, desc.zeta)
    colptr = np.arange(0, h * desc.zeta + 1, desc.zeta)
    return sp.csc_matrix((signs.ravel() / np.sqrt(desc.zeta), rows.ravel(), colptr),
                         shape=(desc.s, h))


class SRTT:
    """S = sqrt(h/s) D F E of eq. (sketching_trig): E = diag(signs), F = orthonormal DCT-II of
    length h (scipy.fft.dct, norm="ortho"), D = the rows ``rows`` of the identity.  Applied as
    S v = sqrt(h/s) (F (E v))[rows]; the transpose S^T u = sqrt(h/s) E F^T (D^T u)."""

    def __init__(self, signs, rows):
        self.signs, self.rows = signs, rows
        self.h, self.s = len(signs), len(rows)
        self.shape = (self.s, self.h)
        self.scale = np.sqrt(self.h / self.s)

    def __matmul__(self, v):
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 2:
            return np.stack([self @ v[:, j] for j in range(v.shape[1])], axis=1)
        return self.scale * scipy.fft.dct(self.signs * v, type=2, norm="ortho")[self.rows]

    @property
    def T(self):
        outer = self

        class _T:
            shape = (outer.h, outer.s)

            def __matmul__(self, u):
                full = np.zeros(outer.h)
                full[outer.rows] = u
                return outer.scale * outer.signs * scipy.fft.idct(full, type=2, norm="ortho")

        return _T()

    def toarray(self):
        return np.stack([self @ e for e in np.eye(self.h)], axis=1)


# -------------------------------------------------------------------------- operators

class _Op:
    def __init__(self, rows, cols, fwd, adj):
        self.shape = (rows, cols)
        self.apply = fwd
        self.adjoint = adj


def _conv2d(psf, nx, ny):
    """A x = 2D convolution with psf, zero boundary, same size: out[i,j] = sum psf[a,c] x[i-a+kh//2, j-c+kw//2]."""
    kh, kw = psf.shape
    P = np.asarray(psf, dtype=np.float64)

    def fwd(x):
        img = x.reshape(ny, nx)
        out = np.zeros((ny, nx))
        for a in range(kh):
            for c in range(kw):
                da, dc = a - kh // 2, c - kw // 2        # out[i, j] += P[a, c] * img[i - da, j - dc]
                i0, i1 = max(0, da), min(ny, ny + da)
                j0, j1 = max(0, dc), min(nx, nx + dc)
                if i0 < i1 and j0 < j1:
                    out[i0:i1, j0:j1] += P[a, c] * img[i0 - da:i1 - da, j0 - dc:j1 - dc]
        return out.ravel()

    def adj(y):
        img = y.reshape(ny, nx)
        out = np.zeros((ny, nx))
        for a in range(kh):
            for c in range(kw):
                da, dc = a - kh // 2, c - kw // 2        # out[i, j] += P[a, c] * img[i + da, j + dc]
                i0, i1 = max(0, -da), min(ny, ny - da)
                j0, j1 = max(0, -dc), min(nx, nx - dc)
                if i0 < i1 and j0 < j1:
                    out[i0:i1, j0:j1] += P[a, c] * img[i0 + da:i1 + da, j0 + dc:j1 + dc]
        return out.ravel()

    return _Op(nx * ny, nx * ny, fwd, adj)


def _fd_axis(x, axis):
    """Forward differences x[k+1] - x[k] along one axis (the rows [-1 1] of D)."""
    return np.diff(x, axis=axis)


def _fd_axis_adj(d, axis, n):
    """D^T applied along one axis: (D^T d)[k] = d[k-1] - d[k] with d[-1] = d[n-1] = 0."""
    shape = list(d.shape)
    shape[axis] = n
    out = np.zeros(shape)
    sl = [slice(None)] * d.ndim
    sl[axis] = slice(0, n - 1)
    out[tuple(sl)] -= d
    sl[axis] = slice(1, n)
    out[tuple(sl)] += d
    return out


def _reg(L):
    nx, ny, nt = L.nx, L.ny, L.nt
    if L.kind == "fd1":
        return _Op(nx - 1, nx, lambda x: _fd_axis(x, 0), lambda d: _fd_axis_adj(d, 0, nx))
    if L.kind == "grad2d":
        nh = ny * (nx - 1)

        def fwd(x):
            img = x.reshape(ny, nx)
            return np.concatenate([_fd_axis(img, 1).ravel(), _fd_axis(img, 0).ravel()])

        def adj(d):
            h = d[:nh].reshape(ny, nx - 1)
            v = d[nh:].reshape(ny - 1, nx)
            return (_fd_axis_adj(h, 1, nx) + _fd_axis_adj(v, 0, ny)).ravel()

        return _Op(L.p, nx * ny, fwd, adj)
    if L.kind == "laplace2d":
        def lap(x):
            img = x.reshape(ny, nx)
            out = 4.0 * img
            out[1:, :] -= img[:-1, :]
            out[:-1, :] -= img[1:, :]
            out[:, 1:] -= img[:, :-1]
            out[:, :-1] -= img[:, 1:]
            return out.ravel()
        return _Op(nx * ny, nx * ny, lap, lap)
    if L.kind == "spacetime":
        n1 = nt * ny * (nx - 1)
        n2 = nt * (ny - 1) * nx

        def fwd(x):
            vol = x.reshape(nt, ny, nx)
            return np.concatenate([_fd_axis(vol, 2).ravel(), _fd_axis(vol, 1).ravel(),
                                   _fd_axis(vol, 0).ravel()])

        def adj(d):
            a = d[:n1].reshape(nt, ny, nx - 1)
            b = d[n1:n1 + n2].reshape(nt, ny - 1, nx)
            c = d[n1 + n2:].reshape(nt - 1, ny, nx)
            return (_fd_axis_adj(a, 2, nx) + _fd_axis_adj(b, 1, ny) + _fd_axis_adj(c, 0, nt)).ravel()

        return _Op(L.p, nx * ny * nt, fwd, adj)
    raise ValueError(L.kind)


def make_operators(problem):
    """(A, L) as objects with .apply / .adjoint / .shape, in float64."""
    A = problem.A
    if A.kind == "dense":
        M = np.asarray(A.dense, dtype=np.float64)
        Aop = _Op(A.m, A.n, lambda x: M @ x, lambda y: M.T @ y)
    elif A.kind == "csr":
        M = sp.csr_matrix((A.val.astype(np.float64), A.col, A.row_ptr), shape=(A.m, A.n))
        MT = M.T.tocsr()
        Aop = _Op(A.m, A.n, lambda x: M @ x, lambda y: MT @ y)
    elif A.kind == "conv2d":
        Aop = _conv2d(A.psf, A.nx, A.ny)
    else:
        raise ValueError(A.kind)
    return Aop, _reg(problem.L)


def tikhonov_functional(Aop, Lop, b, lam, x):
    """J(x) = ||A x - b||^2 + lam ||L x||^2 (eq. tik)."""
    return float(np.sum((Aop.apply(x) - b) ** 2) + lam * np.sum(Lop.apply(x) ** 2))


def gradient(Aop, Lop, b, lam, x):
    """r = A^T (A x - b) + lam L^T (L x) (eq. gradient, with x = V_k y_k)."""
    return Aop.adjoint(Aop.apply(x) - b) + lam * Lop.adjoint(Lop.apply(x))


def dense_matrix(op, n):
    return np.stack([op.apply(e) for e in np.eye(n)], axis=1)


def direct_solve(Aop, Lop, b, lam, SA=None, SL=None):
    """argmin_x ||S_A (A x - b)||^2 + lam ||S_L L x||^2 by a dense least-squares solve (tiny n)."""
    n = Aop.shape[1]
    A = dense_matrix(Aop, n)
    L = dense_matrix(Lop, n)
    bb = b
    if SA is not None:
        SAd = SA.toarray() if sp.issparse(SA) else SA
        A, bb = SAd @ A, SAd @ b
    if SL is not None:
        SLd = SL.toarray() if sp.issparse(SL) else SL
        L = SLd @ L
    M = np.vstack([A, np.sqrt(lam) * L])
    rhs = np.concatenate([bb, np.zeros(L.shape[0])])
    return np.linalg.lstsq(M, rhs, rcond=None)[0]


# --------------------------------------------------------------------- building blocks

def initial_basis(Aop, b, ell=3):
    """V_0: orthonormal basis of the Krylov space K_l(A^T A, A^T b) (Sec. 2.1; l = 3 in Sec. 4)."""
    v = Aop.adjoint(b)
    V = [v / np.linalg.norm(v)]
    for _ in range(1, ell):
        w = Aop.adjoint(Aop.apply(V[-1]))
        Vm = np.stack(V, axis=1)
        for _pass in range(2):
            w = w - Vm @ (Vm.T @ w)
        V.append(w / np.linalg.norm(w))
    return np.stack(V, axis=1)


def qr_append(Q, R, u, passes=2, breakdown_tol=1e-13):
    """Append the column u to the thin QR factorisation Q R (eq. updqr).

    p = Q^T u; r_perp = u - Q p; rho = ||r_perp||; q_new = r_perp / rho; R gains the column
    [p; rho].  With passes = 2 the projection is repeated on r_perp and the two coefficient
    vectors are added (classical Gram-Schmidt twice).  If rho <= breakdown_tol * ||u|| the
    new direction is treated as numerically dependent: rho = 0 and q_new = 0.
    Returns (Q', R', rho, broke_down).
    """
    h, d = Q.shape
    v = np.array(u, dtype=np.float64, copy=True)
    p = np.zeros(d)
    for _ in range(passes):
        c = Q.T @ v
        v = v - Q @ c
        p = p + c
    rho = float(np.linalg.norm(v))
    broke = rho <= breakdown_tol * float(np.linalg.norm(u))
    if broke:
        rho = 0.0
        q = np.zeros(h)
    else:
        q = v / rho
    R2 = np.zeros((d + 1, d + 1))
    R2[:d, :d] = R
    R2[:d, d] = p
    R2[d, d] = rho
    return np.concatenate([Q, q[:, None]], axis=1), R2, rho, broke


def projected_solve(RA, RL, dA, lam):
    """y = argmin || [R_A; sqrt(lam) R_L] y - [d_A; 0] || (eq. projected_sketched_bis).

    Householder QR of the stacked 2d x d matrix from scratch, then back substitution.
    Returns (y, T) with T the triangular factor (T^T T = R_A^T R_A + lam R_L^T R_L).
    """
    d = RA.shape[0]
    M = np.vstack([RA, np.sqrt(lam) * RL])
    rhs = np.concatenate([dA, np.zeros(d)])
    Qs, T = np.linalg.qr(M)
    y = scipy.linalg.solve_triangular(T, Qs.T @ rhs, lower=False)
    return y, T


def combine(W, y):
    """x = W y, the iterate of Algorithm 2 from its projected coefficients (a matmul).  A
    module-level step so that the floor model of the parity tests can perturb its terms."""
    return W @ y


def refine_step(Aop, Lop, b, lam, W, y, T):
    """One refinement step of the projected problem, sketched preconditioner, no inner solve.

    With the stacked operator M = [A W; sqrt(lam) L W] and right-hand side [b; 0], the
    correction is dy = (T^T T)^{-1} M^T ([b; 0] - M y) = -(T^T T)^{-1} W^T r(y), where
    r(y) = A^T (A W y - b) + lam L^T L W y is the gradient of eq. (gradient) and T the
    triangular factor of the sketched problem.  Its fixed point is the unsketched
    projected solution of eq. (sGKS_noSASL).
    """
    x = combine(W, y)
    g = W.T @ gradient(Aop, Lop, b, lam, x)
    t = scipy.linalg.solve_triangular(T, g, trans="T", lower=False)
    return y - scipy.linalg.solve_triangular(T, t, lower=False)


# ------------------------------------------------------------------------------- solvers

def sgks(problem, iters=None, n_refine=None, sketched=True, cgs_passes=2, tol=0.0,
         W0=None, record_x=False, record_state=False):
    """Algorithm 2 (sGKS); with sketched=False the projected solve is eq. (sGKS_noSASL) (sGKS_0).

    Loop: W_0 = V_0 (orthonormal Krylov basis, range W_0 = range V_0 as Proposition 1
    assumes); the QR factors of S_A A W_0 and S_L L W_0 are built by appending W_0's
    columns; then y_0 and x_0 = W_0 y_0.  Each iteration k = 1..iters:
      r_k = A^T (A x_{k-1} - b) + lam L^T L x_{k-1}  (eq. gradient), W_k = [W_{k-1}, r_k]
      (no normalisation, no reorthogonalisation); append S_A A r_k and S_L L r_k to the
      sketched QR factors (eq. updqr) and q_new^T S_A b to d_A (eq. dA_update);
      y_k from eq. (projected_sketched_bis); n_refine refinement steps; x_k = W_k y_k;
      RC_k = ||x_k - x_{k-1}|| / ||x_{k-1}|| (eq. RC); stop if tol > 0 and RC_k < tol.
    Returns a dict with x, y, W, the factors and the per-iteration RC / RRE records.
    """
    P = problem
    iters = P.iters if iters is None else iters
    n_refine = P.n_refine if n_refine is None else n_refine
    Aop, Lop = make_operators(P)
    b = np.asarray(P.b, dtype=np.float64)
    lam = float(P.lam)
    if sketched:
        SA = sketch_operator(P.sketch, 0, P.m)
        SL = sketch_operator(P.sketch, 1, P.p)
        sA = lambda v: SA @ v  # noqa: E731
        sL = lambda v: SL @ v  # noqa: E731
    else:
        sA = sL = lambda v: v  # noqa: E731
    Sb = sA(b)
    W = initial_basis(Aop, b, P.ell) if W0 is None else np.array(W0, dtype=np.float64)
    hA, hL = len(Sb), len(sL(np.zeros(P.p)))
    QA, RA = np.zeros((hA, 0)), np.zeros((0, 0))
    QL, RL = np.zeros((hL, 0)), np.zeros((0, 0))
    dA = np.zeros(0)
    breakdowns = 0

    def append(w):
        nonlocal QA, RA, QL, RL, dA, breakdowns
        QA, RA, _, bA = qr_append(QA, RA, sA(Aop.apply(w)), cgs_passes)
        QL, RL, _, bL = qr_append(QL, RL, sL(Lop.apply(w)), cgs_passes)
        dA = np.concatenate([dA, [QA[:, -1] @ Sb]])
        breakdowns += int(bA and bL)

    for j in range(W.shape[1]):
        append(W[:, j])

    def solve():
        # the projected solve and its refinement steps; returns y_k and the chain y^0 .. y^R
        y, T = projected_solve(RA, RL, dA, lam)
        chain = [y]
        for _ in range(n_refine):
            y = refine_step(Aop, Lop, b, lam, W, y, T)
            chain.append(y)
        return y, chain

    xt = np.asarray(P.x_true, dtype=np.float64)
    nxt = np.linalg.norm(xt)
    y, chain = solve()
    x = combine(W, y)
    rc, rre, xs = [], [np.linalg.norm(x - xt) / nxt], [x.copy()] if record_x else None
    ys = [y.copy()] if record_x else None
    yrs = [[c.copy() for c in chain]] if record_x else None
    for k in range(1, iters + 1):
        r = gradient(Aop, Lop, b, lam, x)
        W = np.concatenate([W, r[:, None]], axis=1)
        append(r)
        y, chain = solve()
        x_new = combine(W, y)
        rc.append(np.linalg.norm(x_new - x) / np.linalg.norm(x))
        rre.append(np.linalg.norm(x_new - xt) / nxt)
        x = x_new
        if record_x:
            xs.append(x.copy())
            ys.append(y.copy())
            yrs.append([c.copy() for c in chain])
        if tol > 0 and rc[-1] < tol:
            break
    out = dict(x=x, y=y, W=W, rc=np.array(rc), rre=np.array(rre), breakdowns=breakdowns,
               iters=k if iters > 0 else 0)
    if record_x:
        out["xs"] = xs
        out["ys"] = ys
        out["yrs"] = yrs   # per iteration: y before refinement, then after each refinement step
    if record_state:
        out.update(QA=QA, RA=RA, QL=QL, RL=RL, dA=dA, Sb=Sb)
    return out


def gks(problem, iters=None, tau=1e-10, cgs_passes=2, tol=0.0, record_x=False):
    """Algorithm 1 (GKS): orthonormal V_k, QR updates of A V_k and L V_k, eq. (projected_withQR).

    Each iteration: r_{k+1} from eq. (gradient); v~ = (I - V V^T) r_{k+1}; loss ratio
    ||V^T v~|| / ||v~|| (eq. loss_criterion); if >= tau a second projection; normalise and
    append.  Stopping test ||y_k - [y_{k-1}; 0]|| <= tol (eq. stoppingcriterion_cheap) when tol > 0.
    """
    P = problem
    iters = P.iters if iters is None else iters
    Aop, Lop = make_operators(P)
    b = np.asarray(P.b, dtype=np.float64)
    lam = float(P.lam)
    V = initial_basis(Aop, b, P.ell)
    QA, RA = np.zeros((P.m, 0)), np.zeros((0, 0))
    QL, RL = np.zeros((P.p, 0)), np.zeros((0, 0))
    dA = np.zeros(0)

    def append(v):
        nonlocal QA, RA, QL, RL, dA
        QA, RA, _, _ = qr_append(QA, RA, Aop.apply(v), cgs_passes)
        QL, RL, _, _ = qr_append(QL, RL, Lop.apply(v), cgs_passes)
        dA = np.concatenate([dA, [QA[:, -1] @ b]])

    for j in range(V.shape[1]):
        append(V[:, j])
    xs = []
    y_prev = None
    second_passes = 0
    for k in range(0, iters + 1):
        y, _ = projected_solve(RA, RL, dA, lam)
        x = V @ y
        if record_x:
            xs.append(x.copy())
        if k > 0 and tol > 0 and np.linalg.norm(y - np.concatenate([y_prev, [0.0]])) <= tol:
            break
        if k == iters:
            break
        r = gradient(Aop, Lop, b, lam, x)
        v = r - V @ (V.T @ r)
        loss = np.linalg.norm(V.T @ v) / np.linalg.norm(v)
        if loss >= tau:
            v = v - V @ (V.T @ v)
            second_passes += 1
        v = v / np.linalg.norm(v)
        V = np.concatenate([V, v[:, None]], axis=1)
        append(v)
        y_prev = y
    out = dict(x=x, y=y, V=V, RA=RA, RL=RL, second_passes=second_passes)
    if record_x:
        out["xs"] = xs
    return out
