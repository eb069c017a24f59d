"""Straight-ray intersection-length matrices (Siddon's method), vectorised in NumPy.

Siddon (Med. Phys. 12, 1985) computes the exact length of a line segment inside each pixel
of a regular grid by merging the parameters at which the segment crosses the vertical and
horizontal grid lines.  This is input generation only: the result is a CSR matrix whose
entry (ray r, pixel j) is the length of ray r inside pixel j; both the oracle and the CUDA
library read the same arrays.

Grid: N x N pixels of unit size covering [0, N]^2; pixel (iy, ix) covers
[ix, ix+1] x [iy, iy+1] and has column index iy*N + ix.
"""
from __future__ import annotations

import numpy as np


def trace_segments(p0: np.ndarray, p1: np.ndarray, N: int, min_len: float = 1e-9):
    """Trace segments p0[r] -> p1[r] (shape (R, 2), (x, y) in pixel units) through the grid.

    Returns (counts, cols, vals): counts[r] = nnz of ray r; cols/vals concatenated over rays,
    columns ascending within each ray, values float64 lengths.
    """
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    R = p0.shape[0]
    d = p1 - p0
    seglen = np.hypot(d[:, 0], d[:, 1])
    ks = np.arange(N + 1, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        # parameters of the crossings with x = k and y = k (t in [0, 1] along the segment)
        tx = (ks[None, :] - p0[:, 0:1]) / d[:, 0:1]
        ty = (ks[None, :] - p0[:, 1:2]) / d[:, 1:2]
        # entry / exit of the square [0, N]^2 (slab method)
        tx0 = np.where(d[:, 0] != 0, np.minimum(tx[:, 0], tx[:, N]), -np.inf)
        tx1 = np.where(d[:, 0] != 0, np.maximum(tx[:, 0], tx[:, N]), np.inf)
        ty0 = np.where(d[:, 1] != 0, np.minimum(ty[:, 0], ty[:, N]), -np.inf)
        ty1 = np.where(d[:, 1] != 0, np.maximum(ty[:, 0], ty[:, N]), np.inf)
    # a segment parallel to an axis must lie inside that slab
    inside_x = (d[:, 0] != 0) | ((p0[:, 0] >= 0) & (p0[:, 0] <= N))
    inside_y = (d[:, 1] != 0) | ((p0[:, 1] >= 0) & (p0[:, 1] <= N))
    t_lo = np.maximum(np.maximum(tx0, ty0), 0.0)
    t_hi = np.minimum(np.minimum(tx1, ty1), 1.0)
    hit = inside_x & inside_y & (t_hi > t_lo)
    t_lo = np.where(hit, t_lo, 0.0)
    t_hi = np.where(hit, t_hi, 0.0)
    tx = np.where(np.isfinite(tx), tx, t_lo[:, None])
    ty = np.where(np.isfinite(ty), ty, t_lo[:, None])
    allt = np.concatenate([t_lo[:, None], t_hi[:, None], tx, ty], axis=1)
    allt = np.clip(allt, t_lo[:, None], t_hi[:, None])
    allt.sort(axis=1)
    lens = np.diff(allt, axis=1) * seglen[:, None]
    tm = 0.5 * (allt[:, 1:] + allt[:, :-1])
    mx = p0[:, 0:1] + tm * d[:, 0:1]
    my = p0[:, 1:2] + tm * d[:, 1:2]
    ix = np.floor(mx).astype(np.int64)
    iy = np.floor(my).astype(np.int64)
    ok = (lens > min_len) & (ix >= 0) & (ix < N) & (iy >= 0) & (iy < N)
    rows = np.broadcast_to(np.arange(R)[:, None], ok.shape)[ok]
    cols = (iy * N + ix)[ok]
    vals = lens[ok]
    # order by (ray, column) and merge any duplicate (ray, pixel) pairs
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size:
        key = rows * (N * N) + cols
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        idx = np.flatnonzero(first)
        vals = np.add.reduceat(vals, idx)
        rows, cols = rows[idx], cols[idx]
    counts = np.bincount(rows, minlength=R)
    return counts, cols, vals


def assemble_csr(chunks, n_cols: int):
    """Concatenate per-chunk (counts, cols, vals) into int32/int32/float32 CSR arrays."""
    counts = np.concatenate([c[0] for c in chunks])
    row_ptr = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    col = np.concatenate([c[1] for c in chunks]).astype(np.int32)
    val = np.concatenate([c[2] for c in chunks]).astype(np.float32)
    assert col.size == row_ptr[-1]
    assert col.size == 0 or (col.min() >= 0 and col.max() < n_cols)
    return row_ptr.astype(np.int32), col, val


def parallel_beam_csr(N: int, angles_deg, nbins: int, spacing: float = 1.0):
    """Parallel-beam projection matrix: one ray per (angle, detector bin), angle-major rows.

    Ray (theta, u): the line {p : (p - c) . (cos theta, sin theta) = u} through the image
    centre c = (N/2, N/2), detector offsets u = (t - (nbins-1)/2) * spacing, t = 0..nbins-1.
    """
    c = N / 2.0
    half = N * 0.75 + 2.0          # half-length of the traced segment: longer than the diagonal
    u = (np.arange(nbins) - (nbins - 1) / 2.0) * spacing
    chunks = []
    for th in np.deg2rad(np.asarray(angles_deg, dtype=np.float64)):
        nrm = np.array([np.cos(th), np.sin(th)])
        dirv = np.array([-np.sin(th), np.cos(th)])
        centre = c + u[:, None] * nrm[None, :]
        p0 = centre - half * dirv[None, :]
        p1 = centre + half * dirv[None, :]
        chunks.append(trace_segments(p0, p1, N))
    return assemble_csr(chunks, N * N)


def chord_length_parallel(N: int, theta_rad: float, u: float) -> float:
    """Closed-form length of the line (theta, u) inside the square [0, N]^2 (centre N/2)."""
    c = N / 2.0
    nrm = np.array([np.cos(theta_rad), np.sin(theta_rad)])
    dirv = np.array([-np.sin(theta_rad), np.cos(theta_rad)])
    p = c + u * nrm
    lo, hi = -np.inf, np.inf
    for k in range(2):
        if abs(dirv[k]) < 1e-300:
            if not (0.0 <= p[k] <= N):
                return 0.0
            continue
        a = (0.0 - p[k]) / dirv[k]
        b = (N - p[k]) / dirv[k]
        lo, hi = max(lo, min(a, b)), min(hi, max(a, b))
    return max(0.0, hi - lo)


def point_rays_csr(N: int, sources: np.ndarray, receivers: np.ndarray):
    """Straight rays from every source to every receiver (source-major rows)."""
    chunks = []
    for s in sources:
        p0 = np.broadcast_to(s, receivers.shape)
        chunks.append(trace_segments(p0, receivers, N))
    return assemble_csr(chunks, N * N)
