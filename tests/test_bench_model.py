"""bench.py's algorithmic byte model: a pass over a stored CSR operator counts its column indices,
values and row pointers once; the matrix-free convolution adds nothing; classes that do not
apply A (the combine, the small phase) are the same for both."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import small_problem  # noqa: E402


def test_csr_passes_count_the_matrix():
    P = small_problem("seismic2d")
    nnz = len(P.A.col)
    for T in (4, 8):
        at = bench.bytes_model(P, "gradient_append", 20, T) - bench._vector_bytes(P.n, P.m, P.sketch.s, 20, T,
                                                                                   "gradient_append")
        assert at == nnz * (4 + T) + (P.n + 1) * 4          # the stored transpose: n rows
        a = bench.bytes_model(P, "sketch_column", 20, T) - bench._vector_bytes(P.n, P.m, P.sketch.s, 20, T,
                                                                                "sketch_column")
        assert a == nnz * (4 + T) + (P.m + 1) * 4           # A itself: m rows
        assert bench.bytes_model(P, "combine", 20, T) == bench._vector_bytes(P.n, P.m, P.sketch.s, 20, T, "combine")


def test_convolution_is_matrix_free():
    P = small_problem("deblur2d")
    for cls in ("gradient_append", "sketch_column", "gradient_refine"):
        assert bench.bytes_model(P, cls, 10, 4) == bench._vector_bytes(P.n, P.m, P.sketch.s, 10, 4, cls)


def test_labels_follow_the_config():
    P = small_problem("ct2d")
    metric, wl = bench.labels("ct2d", P)
    assert "ct2d" in metric and wl.startswith("ct2d: A CSR")
    assert bench.labels("deblur2d") == (bench.METRIC, bench.WORKLOAD)


def test_batch_byte_model():
    """Batched passes: the CSR arrays once per pass for all B instances, the instance vectors once
    each; basis values 8 bytes in the FP64 and float-float forms, 4 in the FP32 forms."""
    B, n, m, nnz, d = 64, 1000, 700, 50000, 20.0
    a_ff = bench.batch_bytes("apply_column", B, n, m, nnz, d, "ff")
    a_32 = bench.batch_bytes("apply_column", B, n, m, nnz, d, "fp32")
    assert a_ff == nnz * 8 + (m + 1) * 4 + B * (n * 8 + m * 8)
    assert a_ff - a_32 == B * n * 4
    g = bench.batch_bytes("gradient_append", B, n, m, nnz, d, "fp64")
    assert g == nnz * 8 + (n + 1) * 4 + B * (m * 8 + n * 8 + n * 8)
    c = bench.batch_bytes("combine", B, n, m, nnz, d, "ff")
    assert c == B * (d * (n + m) * 8 + n * 8 * 4 + m * 8 * 2)
