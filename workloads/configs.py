"""The five synthetic workloads and small test-sized variants.

Each generator is seeded (NumPy PCG64) and returns a :class:`Problem`.  Recipes:

deconv1d  (1D deconvolution, plain FP64): n = m = 256; A dense Toeplitz Gaussian blur,
          A_ij = exp(-(i-j)^2 / (2*3^2)) for |i-j| <= 12, rows normalised to sum 1;
          L = D_256 (255 x 256); x_true piecewise constant with 5 pieces (4 sorted
          breakpoints uniform in [1, 255], values U[0,1]); 1% noise; lambda = 1e-2;
          30 iterations; Gaussian sketch with s = 120 rows; seed 0.
deblur2d  (image deblurring, after Experiment 1, Sec. 4.1): 256 x 256 image; A = 2D convolution with a
          9x9 Gaussian PSF, sigma = 2, zero boundary; L = 2D forward-difference gradient;
          x_true = 20 axis-aligned rectangles (later ones overwrite), intensities U[0,1];
          1% noise; lambda = 5e-3; 100 iterations; sparse-sign sketch, zeta = 8, s = 400;
          FP32 operators with 2 refinement steps.
ct2d      (parallel-beam X-ray CT, after Experiment 2, Sec. 4.2.1): 512 x 512 image; 180 angles j*1 deg,
          725 detector bins of 1 px; A = CSR of ray-pixel intersection lengths (float32
          values, int32 indices); phantom = 10 random ellipses, densities U[0,1], added;
          L = grad2d; 2% noise; instance i of the 64-instance batch has noise seed i and
          lambda_i = 10^(-4 + 3 i / 63); 150 iterations; sparse-sign, zeta = 8, s = 600.
seismic2d (travel-time tomography, after Experiment 3, Sec. 4.2.2): 256 x 256 slowness grid; 64 sources on
          the left edge, 128 receivers (64 on the right edge, 64 on the top edge), m = 8192
          straight rays; x_true = 1 + 0.1 * (Gaussian random field, correlation length 20
          cells, unit std); L = 5-point Laplacian; 1% noise; 80 iterations; sparse-sign,
          zeta = 8, s = 400.
dynct     (dynamic CT, after Experiment 4, Sec. 4.3): 128 x 128 x F frames (F = 32 by default); frame t
          sees 30 angles (6 t + 0.2 j) deg mod 180, j = 0..29, 185 bins; A = block-diagonal
          CSR; L = Psi (eq. spacetime_tik); 4 ellipses moving 1 or 2 px per frame; 1% noise;
          200 iterations; sparse-sign, zeta = 8, s = 800; FP32 operators with 3 refinement
          steps.

The noise vector is scaled so that ||e|| / ||A x_true|| equals the stated level exactly
(Sec. 4: sigma = ||e|| / ||A x||).  Every array that defines the problem is rounded to
float32 so that both solver precisions see the same problem.
"""
from __future__ import annotations

import numpy as np
import scipy.signal
import scipy.sparse as sp

from .problem import OperatorDesc, Problem, RegDesc, SketchDesc
from .raytrace import parallel_beam_csr, point_rays_csr

CONFIG_NAMES = ("deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct")

# lambda for the configs that do not state one, chosen by a grid search of 15 log-spaced
# values with the FP64 oracle on the seed-0 instance (minimum RRE), as in Sec. 4 (lambda*
# hand-tuned to minimise the RRE).
LAMBDA_SEISMIC = 2.683
LAMBDA_DYNCT = 26.83


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _apply_A(A: OperatorDesc, x: np.ndarray) -> np.ndarray:
    """Forward model used to synthesise data only."""
    if A.kind == "dense":
        return A.dense @ x
    if A.kind == "csr":
        M = sp.csr_matrix((A.val.astype(np.float64), A.col, A.row_ptr), shape=(A.m, A.n))
        return M @ x
    if A.kind == "conv2d":
        img = x.reshape(A.ny, A.nx)
        return scipy.signal.convolve2d(img, A.psf.astype(np.float64), mode="same",
                                       boundary="fill").ravel()
    raise ValueError(A.kind)


def _noisy(A, x_true, level, rng):
    bt = _apply_A(A, x_true)
    g = rng.standard_normal(bt.shape)
    e = level * np.linalg.norm(bt) * g / np.linalg.norm(g)
    return _f32(bt + e)


def _sketch(kind, s, m, p, zeta=8, seed=0):
    if kind == "gaussian":
        SA = _rng(seed, 101).standard_normal((s, m)) / np.sqrt(s)
        SL = _rng(seed, 102).standard_normal((s, p)) / np.sqrt(s)
        return SketchDesc("gaussian", s, zeta, seed, SA=SA, SL=SL)
    if kind == "srtt":
        return srtt_sketch(s, m, p, seed)
    return SketchDesc("sparse_sign", s, zeta, seed)


def srtt_sketch(s, m, p, seed=0):
    """Rademacher signs and s distinct sampled rows for S_A (length m) and S_L (length p)."""
    ra, rl = _rng(seed, 103), _rng(seed, 104)
    return SketchDesc("srtt", s, 0, seed,
                      signs_A=ra.choice(np.array([-1, 1], dtype=np.int8), size=m),
                      rows_A=np.sort(ra.choice(m, size=s, replace=False)).astype(np.int32),
                      signs_L=rl.choice(np.array([-1, 1], dtype=np.int8), size=p),
                      rows_L=np.sort(rl.choice(p, size=s, replace=False)).astype(np.int32))


# ----------------------------------------------------------------------------- operators

def blur1d_dense(n: int, sigma: float = 3.0, trunc: float = 4.0) -> OperatorDesc:
    i = np.arange(n)
    D = np.abs(i[:, None] - i[None, :]).astype(np.float64)
    A = np.where(D <= np.floor(trunc * sigma), np.exp(-D ** 2 / (2 * sigma ** 2)), 0.0)
    A /= A.sum(axis=1, keepdims=True)
    return OperatorDesc("dense", n, n, dense=_f32(A))


def gaussian_psf(k: int, sigma: float) -> np.ndarray:
    r = np.arange(k) - k // 2
    h = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2 * sigma ** 2))
    return (h / h.sum()).astype(np.float32)


def conv2d_op(nx: int, ny: int, psf: np.ndarray) -> OperatorDesc:
    return OperatorDesc("conv2d", nx * ny, nx * ny, nx=nx, ny=ny, psf=np.asarray(psf, np.float32))


def ct_op(N: int, angles_deg, nbins: int) -> OperatorDesc:
    rp, col, val = parallel_beam_csr(N, angles_deg, nbins)
    return OperatorDesc("csr", len(rp) - 1, N * N, row_ptr=rp, col=col, val=val, nx=N, ny=N)


def blockdiag_csr(blocks):
    """blkdiag(A_1, ..., A_F) of CSR OperatorDescs (eq. blockF)."""
    rps, cols, vals = [np.zeros(1, np.int64)], [], []
    off_r = off_c = off_nz = 0
    for B in blocks:
        rps.append(B.row_ptr[1:].astype(np.int64) + off_nz)
        cols.append(B.col.astype(np.int64) + off_c)
        vals.append(B.val)
        off_nz += int(B.row_ptr[-1])
        off_r += B.m
        off_c += B.n
    rp = np.concatenate(rps)
    assert rp[-1] < 2 ** 31
    return OperatorDesc("csr", off_r, off_c, row_ptr=rp.astype(np.int32),
                        col=np.concatenate(cols).astype(np.int32),
                        val=np.concatenate(vals).astype(np.float32), frames=len(blocks))


# ------------------------------------------------------------------------------ phantoms

def phantom_steps(n, rng, pieces=5):
    bp = np.sort(rng.choice(np.arange(1, n), size=pieces - 1, replace=False))
    vals = rng.uniform(0, 1, size=pieces)
    x = np.empty(n)
    edges = np.concatenate([[0], bp, [n]])
    for k in range(pieces):
        x[edges[k]:edges[k + 1]] = vals[k]
    return _f32(x)


def phantom_rectangles(nx, ny, count, rng):
    img = np.zeros((ny, nx))
    for _ in range(count):
        x0, x1 = np.sort(rng.integers(0, nx + 1, size=2))
        y0, y1 = np.sort(rng.integers(0, ny + 1, size=2))
        x1 = max(x1, x0 + 1)
        y1 = max(y1, y0 + 1)
        img[y0:y1, x0:x1] = rng.uniform(0, 1)
    return _f32(img.ravel())


def _ellipse_mask(N, cx, cy, a, b, ang):
    yy, xx = np.mgrid[0:N, 0:N] + 0.5
    dx, dy = xx - cx, yy - cy
    c, s = np.cos(ang), np.sin(ang)
    u = (c * dx + s * dy) / a
    v = (-s * dx + c * dy) / b
    return (u * u + v * v) <= 1.0


def phantom_ellipses(N, count, rng, rmin=10.0, rmax=120.0):
    img = np.zeros((N, N))
    R = 0.4 * N
    for _ in range(count):
        r = R * np.sqrt(rng.uniform())
        t = rng.uniform(0, 2 * np.pi)
        cx, cy = N / 2 + r * np.cos(t), N / 2 + r * np.sin(t)
        a, b = rng.uniform(rmin, rmax, size=2) * (N / 512.0)
        img += rng.uniform(0, 1) * _ellipse_mask(N, cx, cy, a, b, rng.uniform(0, np.pi))
    return _f32(img.ravel())


def phantom_moving_ellipses(N, frames, rng, count=4):
    params = []
    for _ in range(count):
        cx, cy = rng.uniform(0.3 * N, 0.7 * N, size=2)
        a, b = rng.uniform(0.06 * N, 0.16 * N, size=2)
        ang = rng.uniform(0, np.pi)
        speed = float(rng.choice([1.0, 2.0]))
        th = rng.uniform(0, 2 * np.pi)
        params.append((cx, cy, a, b, ang, speed * np.cos(th), speed * np.sin(th), rng.uniform(0, 1)))
    vol = np.zeros((frames, N, N))
    for t in range(frames):
        for (cx, cy, a, b, ang, vx, vy, dens) in params:
            vol[t] += dens * _ellipse_mask(N, cx + vx * t, cy + vy * t, a, b, ang)
    return _f32(vol.ravel())


def gaussian_random_field(N, corr_len, rng):
    w = rng.standard_normal((N, N))
    k = np.fft.fftfreq(N)
    kk = k[:, None] ** 2 + k[None, :] ** 2
    sig = corr_len / np.sqrt(2.0)
    filt = np.exp(-2.0 * (np.pi ** 2) * (sig ** 2) * kk)
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    f = (f - f.mean()) / f.std()
    return f.ravel()


# ------------------------------------------------------------------------------- configs

def make_deconv1d(seed=0, n=256, s=120, iters=30, lam=1e-2, level=0.01):
    rng = _rng(seed, 0)
    A = blur1d_dense(n)
    L = RegDesc("fd1", nx=n)
    x = phantom_steps(n, rng)
    b = _noisy(A, x, level, _rng(seed, 1))
    return Problem("deconv1d", A, L, b, x, lam, iters, _sketch("gaussian", s, A.m, L.p, seed=seed),
                   n_refine=0, precision="fp64")


def make_deblur2d(seed=0, N=256, s=400, iters=100, lam=5e-3, level=0.01, n_refine=2,
                  rects=20, zeta=8):
    rng = _rng(seed, 0)
    A = conv2d_op(N, N, gaussian_psf(9, 2.0))
    L = RegDesc("grad2d", nx=N, ny=N)
    x = phantom_rectangles(N, N, rects, rng)
    b = _noisy(A, x, level, _rng(seed, 1))
    return Problem("deblur2d", A, L, b, x, lam, iters, _sketch("sparse_sign", s, A.m, L.p, zeta, seed),
                   n_refine=n_refine, precision="fp32")


def ct_lambda(i, batch=64):
    return float(10.0 ** (-4.0 + 3.0 * i / (batch - 1)))


def make_ct2d(instance=42, seed=0, N=512, n_angles=180, nbins=725, s=600, iters=150,
              level=0.02, zeta=8, ellipses=10, precision="fp32", n_refine=0, A=None):
    rng = _rng(seed, 0)
    if A is None:
        A = ct_op(N, np.arange(n_angles) * (180.0 / n_angles), nbins)
    L = RegDesc("grad2d", nx=N, ny=N)
    x = phantom_ellipses(N, ellipses, rng)
    b = _noisy(A, x, level, _rng(instance, 1))
    return Problem("ct2d", A, L, b, x, ct_lambda(instance), iters,
                   _sketch("sparse_sign", s, A.m, L.p, zeta, seed), n_refine=n_refine,
                   precision=precision, meta={"instance": instance})


def seismic_geometry(N, n_src=64, n_rec_side=64):
    ys = (np.arange(n_src) + 0.5) * (N / n_src)
    src = np.stack([np.zeros(n_src), ys], axis=1)
    t = (np.arange(n_rec_side) + 0.5) * (N / n_rec_side)
    rec_right = np.stack([np.full(n_rec_side, float(N)), t], axis=1)
    rec_top = np.stack([t, np.full(n_rec_side, float(N))], axis=1)
    return src, np.concatenate([rec_right, rec_top], axis=0)


def make_seismic2d(seed=0, N=256, s=400, iters=80, lam=None, level=0.01, zeta=8,
                   corr_len=20.0, precision="fp32", n_refine=0):
    rng = _rng(seed, 0)
    src, rec = seismic_geometry(N)
    rp, col, val = point_rays_csr(N, src, rec)
    A = OperatorDesc("csr", len(rp) - 1, N * N, row_ptr=rp, col=col, val=val, nx=N, ny=N)
    L = RegDesc("laplace2d", nx=N, ny=N)
    x = _f32(1.0 + 0.1 * gaussian_random_field(N, corr_len, rng))
    b = _noisy(A, x, level, _rng(seed, 1))
    return Problem("seismic2d", A, L, b, x, LAMBDA_SEISMIC if lam is None else lam, iters,
                   _sketch("sparse_sign", s, A.m, L.p, zeta, seed), n_refine=n_refine,
                   precision=precision)


def dynct_frame_ops(N=128, frames=32, n_ang=30, nbins=185, step_deg=6.0, sub_deg=0.2):
    ops = []
    for t in range(frames):
        ang = np.mod(step_deg * t + sub_deg * np.arange(n_ang), 180.0)
        ops.append(ct_op(N, ang, nbins))
    return ops


def make_dynct(seed=0, N=128, frames=32, s=800, iters=200, lam=None, level=0.01, zeta=8,
               n_refine=3, precision="fp32", frame_ops=None):
    rng = _rng(seed, 0)
    ops = frame_ops if frame_ops is not None else dynct_frame_ops(N, frames)
    A = blockdiag_csr(ops[:frames])
    L = RegDesc("spacetime", nx=N, ny=N, nt=frames)
    x = phantom_moving_ellipses(N, frames, rng)
    b = _noisy(A, x, level, _rng(seed, 1))
    return Problem("dynct", A, L, b, x, LAMBDA_DYNCT if lam is None else lam, iters,
                   _sketch("sparse_sign", s, A.m, L.p, zeta, seed), n_refine=n_refine,
                   precision=precision, meta={"frames": frames})


def make_problem(name: str, **kw) -> Problem:
    return {
        "deconv1d": make_deconv1d,
        "deblur2d": make_deblur2d,
        "ct2d": make_ct2d,
        "seismic2d": make_seismic2d,
        "dynct": make_dynct,
    }[name](**kw)


def small_problem(kind: str, seed: int = 0, **kw) -> Problem:
    """Reduced sizes of each operator family, for tests that the oracle finishes in seconds.

    kinds: deconv1d (n = 48), deblur2d (24 x 20 image, 5x5 PSF; nx, ny, psf may be given),
    ct2d (32 x 32, 24 angles),
    seismic2d (32 x 32), dynct (16 x 16 x 4 frames), laplace (conv A with Laplacian L).
    """
    if kind == "deconv1d":
        d = dict(n=48, s=40, iters=12)
        d.update(kw)
        return make_deconv1d(seed=seed, **d)
    if kind == "deblur2d":
        rng = _rng(seed, 0)
        nx, ny = kw.pop("nx", 24), kw.pop("ny", 20)
        psf = kw.pop("psf", None)
        A = conv2d_op(nx, ny, gaussian_psf(5, 1.2) if psf is None else psf)
        L = RegDesc("grad2d", nx=nx, ny=ny)
        x = phantom_rectangles(nx, ny, 5, rng)
        b = _noisy(A, x, 0.01, _rng(seed, 1))
        return Problem("deblur2d-small", A, L, b, x, kw.pop("lam", 5e-3), kw.pop("iters", 20),
                       _sketch(kw.pop("sketch", "sparse_sign"), kw.pop("s", 80), A.m, L.p,
                               kw.pop("zeta", 8), seed),
                       n_refine=kw.pop("n_refine", 2), precision=kw.pop("precision", "fp32"))
    if kind == "ct2d":
        N = kw.pop("N", 32)
        A = ct_op(N, np.arange(24) * 7.5, kw.pop("nbins", 47))
        d = dict(N=N, s=80, iters=20, A=A, ellipses=3, precision="fp64")
        d.update(kw)
        return make_ct2d(seed=seed, **d)
    if kind == "seismic2d":
        rng = _rng(seed, 0)
        N = kw.pop("N", 32)
        src, rec = seismic_geometry(N, 16, 16)
        rp, col, val = point_rays_csr(N, src, rec)
        A = OperatorDesc("csr", len(rp) - 1, N * N, row_ptr=rp, col=col, val=val, nx=N, ny=N)
        L = RegDesc("laplace2d", nx=N, ny=N)
        x = _f32(1.0 + 0.1 * gaussian_random_field(N, 4.0, rng))
        b = _noisy(A, x, 0.01, _rng(seed, 1))
        return Problem("seismic2d-small", A, L, b, x, kw.pop("lam", 1.0), kw.pop("iters", 20),
                       _sketch("sparse_sign", kw.pop("s", 80), A.m, L.p, 8, seed),
                       n_refine=kw.pop("n_refine", 0), precision=kw.pop("precision", "fp64"))
    if kind == "dynct":
        N, F = kw.pop("N", 16), kw.pop("frames", 4)
        ops = dynct_frame_ops(N, F, n_ang=6, nbins=23, step_deg=30.0, sub_deg=5.0)
        d = dict(N=N, frames=F, s=100, iters=20, frame_ops=ops, n_refine=1, lam=0.5)
        d.update(kw)
        return make_dynct(seed=seed, **d)
    raise ValueError(kind)
