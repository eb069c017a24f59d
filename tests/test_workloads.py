"""Pins of the synthetic input generators (geometry closed forms, noise level, precision)."""
import numpy as np
import pytest

from workloads import make_problem, small_problem
from workloads.configs import blockdiag_csr, ct_op, seismic_geometry
from workloads.raytrace import chord_length_parallel, parallel_beam_csr, point_rays_csr


def test_parallel_beam_row_sums_equal_chord_lengths():
    N, nb = 32, 47
    angles = np.array([0.0, 7.5, 30.0, 45.0, 90.0, 133.0, 179.0])
    rp, col, val = parallel_beam_csr(N, angles, nb)
    u = np.arange(nb) - (nb - 1) / 2.0
    sums = np.add.reduceat(np.concatenate([val.astype(np.float64), [0]]), rp[:-1])
    sums[np.diff(rp) == 0] = 0.0
    for a, th in enumerate(np.deg2rad(angles)):
        for t in range(nb):
            c = chord_length_parallel(N, th, u[t])
            on_edge = np.isclose(abs(u[t]), N / 2) and np.isclose(np.sin(2 * th), 0)
            if on_edge:
                continue                               # ray along the image border: measure zero
            assert abs(sums[a * nb + t] - c) <= 2e-5 * max(c, 1.0), (a, t)
    assert (val > 0).all() and (val <= np.sqrt(2) + 1e-6).all()


def test_point_rays_row_sums_equal_distances():
    N = 32
    src, rec = seismic_geometry(N, 8, 8)
    rp, col, val = point_rays_csr(N, src, rec)
    sums = np.add.reduceat(val.astype(np.float64), rp[:-1])
    dist = np.linalg.norm(src[:, None, :] - rec[None, :, :], axis=2).ravel()
    assert np.allclose(sums, dist, rtol=2e-6)


def test_csr_columns_sorted_and_unique_within_rows():
    A = small_problem("ct2d").A
    for r in range(A.m):
        c = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert (np.diff(c) > 0).all()


def test_blockdiag_structure():
    ops = [ct_op(8, [0.0, 45.0], 11), ct_op(8, [90.0], 11)]
    B = blockdiag_csr(ops)
    assert B.m == 33 and B.n == 128 and B.frames == 2
    r = 25                                                    # a row of the second block
    assert (B.col[B.row_ptr[r]:B.row_ptr[r + 1]] >= 64).all()


@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_problem_data_is_float32_and_seeded(kind):
    P = small_problem(kind)
    for a in (P.b, P.x_true):
        assert np.array_equal(a, a.astype(np.float32).astype(np.float64))
    Q = small_problem(kind)
    assert np.array_equal(P.b, Q.b)
    assert small_problem(kind, seed=1).b.tolist() != P.b.tolist()


def test_full_size_shapes():
    P = make_problem("deblur2d")
    assert (P.n, P.m, P.p, P.sketch.s, P.iters, P.n_refine) == (65536, 65536, 130560, 400, 100, 2)
    P = make_problem("deconv1d")
    assert (P.n, P.p, P.sketch.s, P.sketch.kind) == (256, 255, 120, "gaussian")
