"""Plain data containers describing one Tikhonov problem min ||Ax-b||^2 + lam ||Lx||^2.

The problem statement is the paper's eq. (tik) in Sec. 1; the sGKS inputs are those of
Algorithm 2 (A, b, L, the two sketches, lambda, the iteration count).  The containers
hold arrays only; applying A or L is the business of the oracle and of the CUDA library.

Conventions shared by every consumer:
  * images are stored row-major with x fastest: pixel (iy, ix) has index iy*nx + ix,
    frames outermost for space-time unknowns (t*ny*nx + iy*nx + ix);
  * all problem data (operator values, b, x_true) are float32-representable, so the
    FP32 and FP64 solver forms solve exactly the same mathematical problem;
  * CSR arrays use int32 row pointers / column indices and float32 values.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class OperatorDesc:
    """Forward operator A (m x n).

    kind = "dense":  ``dense`` holds the (m, n) matrix (row-major, float64 holding float32 values).
    kind = "csr":    ``row_ptr`` (m+1), ``col`` (nnz), ``val`` (nnz, float32).
    kind = "conv2d": 2D convolution of an (ny, nx) image with the odd-sized ``psf`` (kh, kw),
                     zero boundary, output the same size as the input (m = n = nx*ny):
                     (A x)[i, j] = sum_{a, c} psf[a, c] * x[i - a + kh//2, j - c + kw//2].
    ``frames`` > 0 marks a block-diagonal CSR (dynamic CT, eq. blockF) with equal blocks of
    ``m // frames`` rows and ``n // frames`` columns; it is informational only.
    """
    kind: str
    m: int
    n: int
    dense: Optional[np.ndarray] = None
    row_ptr: Optional[np.ndarray] = None
    col: Optional[np.ndarray] = None
    val: Optional[np.ndarray] = None
    nx: int = 0
    ny: int = 0
    psf: Optional[np.ndarray] = None
    frames: int = 0

    @property
    def nnz(self) -> int:
        if self.kind == "csr":
            return int(self.row_ptr[-1])
        if self.kind == "dense":
            return self.m * self.n
        return self.m * int(self.psf.size)


@dataclass
class RegDesc:
    """Regularization operator L (p x n), always a finite-difference stencil.

    kind = "fd1":       first difference D_n in R^{(n-1) x n}, rows [-1 1] (Sec. 4, eq. reg_matrix).
    kind = "grad2d":    [I_ny (x) D_nx ; D_ny (x) I_nx], p = ny(nx-1) + (ny-1)nx (eq. reg_matrix).
    kind = "laplace2d": 5-point Laplacian, zero Dirichlet values outside the grid, p = nx*ny.
    kind = "spacetime": Psi = [I_t (x) I_y (x) D_x ; I_t (x) D_y (x) I_x ; D_t (x) I_y (x) I_x]
                        (Sec. 4.3, eq. spacetime_tik), p = nt(ny(nx-1) + (ny-1)nx) + (nt-1)nx ny.
    """
    kind: str
    nx: int = 0
    ny: int = 1
    nt: int = 1

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nt

    @property
    def p(self) -> int:
        nx, ny, nt = self.nx, self.ny, self.nt
        if self.kind == "fd1":
            return nx - 1
        if self.kind == "grad2d":
            return ny * (nx - 1) + (ny - 1) * nx
        if self.kind == "laplace2d":
            return nx * ny
        if self.kind == "spacetime":
            return nt * (ny * (nx - 1) + (ny - 1) * nx) + (nt - 1) * nx * ny
        raise ValueError(self.kind)


@dataclass
class SketchDesc:
    """The two sketches S_A (s x m) and S_L (s x p) of Sec. 3.

    kind = "sparse_sign": zeta nonzeros +-1/sqrt(zeta) per column, positions and signs from the
                          counter-based hash of (seed, stream, column, draw); stream 0 is S_A,
                          stream 1 is S_L.  Nothing is stored: both sides regenerate it.
    kind = "gaussian":    dense N(0, 1/s) matrices ``SA`` (s x m) and ``SL`` (s x p), drawn here
                          and passed to both sides as inputs.
    kind = "srtt":        the subsampled randomized trigonometric transform of eq.
                          (sketching_trig), S = sqrt(h/s) D F E: E = diag(``signs``) (Rademacher),
                          F the orthonormal DCT-II of length h, D the rows ``rows`` of the identity
                          (s distinct indices).  Signs and rows are drawn here and passed to
                          both sides (``signs_A`` / ``rows_A`` for S_A, ``signs_L`` / ``rows_L``).
    """
    kind: str
    s: int
    zeta: int = 8
    seed: int = 0
    SA: Optional[np.ndarray] = None
    SL: Optional[np.ndarray] = None
    signs_A: Optional[np.ndarray] = None
    rows_A: Optional[np.ndarray] = None
    signs_L: Optional[np.ndarray] = None
    rows_L: Optional[np.ndarray] = None


@dataclass
class Problem:
    name: str
    A: OperatorDesc
    L: RegDesc
    b: np.ndarray
    x_true: np.ndarray
    lam: float
    iters: int
    sketch: SketchDesc
    n_refine: int = 0
    precision: str = "fp64"       # form the config asks for: "fp64" or "fp32" (FP32 operators + FP64 QR/solve)
    ell: int = 3                  # dimension of the initial Krylov subspace (Sec. 4: l = 3)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.n

    @property
    def m(self) -> int:
        return self.A.m

    @property
    def p(self) -> int:
        return self.L.p
