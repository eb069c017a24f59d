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
