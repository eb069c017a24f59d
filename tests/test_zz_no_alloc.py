"""sgks_csr_transpose_noalloc: the CSR transpose for callers that cannot allocate device memory.

Some callers cannot allocate: another allocator may already hold the device memory, or a
service may fix its memory plan at start-up and must not have an allocation fail or stall in
the middle of a request.  This entry point keeps its temporaries in a fixed 16 MiB scratch
array inside the library.  It must give the same transpose, bit for bit, as sgks_csr_transpose,
which allocates its temporaries.  The file is named so that pytest collects it last.  The tests
must pass both alone in a fresh process and after the others.  Two calls in a row, with
different shapes and value types, check that what one call leaves in the shared scratch does
not leak into the next.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from workloads import small_problem

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_18073_gb300 as G
    G.build()
    return G._lib.load()


def _p(t):
    return C.c_void_p(t.data_ptr())


def _transpose(lib, fn, m, n, rp, ci, val):
    """Call one of the two transposes through the C ABI; returns (t_row_ptr, t_col, t_val) on the host."""
    from paper_2606_18073_gb300 import _lib as L
    trp = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    tci = torch.full_like(ci, -7)
    tv = torch.full_like(val, float("nan"))
    vd = L.SGKS_F64 if val.dtype == torch.float64 else L.SGKS_F32
    st = torch.cuda.current_stream().cuda_stream
    rc = getattr(lib, fn)(m, n, int(ci.numel()), _p(rp), _p(ci), _p(val), vd, _p(trp), _p(tci), _p(tv),
                          C.c_void_p(st))
    assert rc == 0, (fn, rc, lib.sgks_last_error(None))
    return trp.cpu().numpy(), tci.cpu().numpy(), tv.cpu().numpy()


def _random_csr(m, n, per_row, dtype, seed):
    """CSR whose rows hold 0 to 2 * per_row distinct sorted columns (5% of them empty), on the device."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 2 * per_row + 1, size=m)
    lens[rng.random(m) < 0.05] = 0
    cols = [np.sort(rng.choice(n, size=k, replace=False)) for k in lens]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate(cols).astype(np.int32)
    val = rng.standard_normal(len(ci))
    return (torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(),
            torch.from_numpy(val).to("cuda", dtype))


def _scratch_need(n, nnz, es):
    a = lambda v: (v + 255) // 256 * 256  # noqa: E731
    return a(4 * (n + 1)) + a(4 * nnz) + a(es * nnz)


def test_noalloc_transpose_matches_allocating_one_twice_in_a_row(lib):
    # call 1: a large FP32 matrix that fills most of the scratch
    m1, n1 = 40000, 65536
    rp, ci, val = _random_csr(m1, n1, 40, torch.float32, seed=11)
    assert 0.5 * SCRATCH_BYTES < _scratch_need(n1, ci.numel(), 4) <= SCRATCH_BYTES
    want = _transpose(lib, "sgks_csr_transpose", m1, n1, rp, ci, val)
    got = _transpose(lib, "sgks_csr_transpose_noalloc", m1, n1, rp, ci, val)
    for g, w in zip(got, want):
        assert np.array_equal(g, w, equal_nan=False)

    # call 2, straight after: a smaller FP64 system matrix (parallel-beam CT rays), so the scratch
    # still holds call 1's counts and rows beyond what this call uses
    P = small_problem("ct2d")
    rp2 = torch.from_numpy(np.ascontiguousarray(P.A.row_ptr, dtype=np.int32)).cuda()
    ci2 = torch.from_numpy(np.ascontiguousarray(P.A.col, dtype=np.int32)).cuda()
    v2 = torch.from_numpy(np.ascontiguousarray(P.A.val, dtype=np.float64)).cuda()
    want2 = _transpose(lib, "sgks_csr_transpose", P.m, P.n, rp2, ci2, v2)
    got2 = _transpose(lib, "sgks_csr_transpose_noalloc", P.m, P.n, rp2, ci2, v2)
    for g, w in zip(got2, want2):
        assert np.array_equal(g, w)


def test_noalloc_transpose_leaves_device_memory_unchanged(lib):
    """After a warm-up call (which may make the library's module resident on the device), a second
    call changes neither the device's free memory nor torch's allocator state: nothing is
    allocated, not even temporarily from a pool that would keep it reserved."""
    from paper_2606_18073_gb300 import _lib as L
    m, n = 20000, 30000
    rp, ci, val = _random_csr(m, n, 30, torch.float32, seed=5)
    _transpose(lib, "sgks_csr_transpose_noalloc", m, n, rp, ci, val)          # warm-up
    out = [torch.empty(n + 1, dtype=torch.int32, device="cuda"), torch.empty_like(ci), torch.empty_like(val)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.sgks_csr_transpose_noalloc(m, n, int(ci.numel()), _p(rp), _p(ci), _p(val), L.SGKS_F32, _p(out[0]),
                                        _p(out[1]), _p(out[2]), C.c_void_p(st))
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


@pytest.mark.parametrize("fn", ["sgks_csr_transpose", "sgks_csr_transpose_noalloc"])
def test_transposes_reject_a_column_outside_the_matrix(lib, fn):
    """A column index outside [0, n) is skipped by the kernels' bounds checks and reported."""
    from paper_2606_18073_gb300 import _lib as L
    m, n = 500, 400
    rp, ci, val = _random_csr(m, n, 6, torch.float64, seed=9)
    orig = int(ci[7])
    ci[7] = n + 3
    trp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    tci, tv = torch.zeros_like(ci), torch.zeros_like(val)
    st = torch.cuda.current_stream().cuda_stream
    rc = getattr(lib, fn)(m, n, int(ci.numel()), _p(rp), _p(ci), _p(val), L.SGKS_F64, _p(trp), _p(tci), _p(tv),
                          C.c_void_p(st))
    assert rc == L.SGKS_ERR_INVALID
    assert b"outside" in lib.sgks_last_error(None)
    ci[7] = orig   # the flag does not outlive the call: the valid matrix transposes cleanly
    rc = getattr(lib, fn)(m, n, int(ci.numel()), _p(rp), _p(ci), _p(val), L.SGKS_F64, _p(trp), _p(tci), _p(tv),
                          C.c_void_p(st))
    assert rc == 0


def test_noalloc_transpose_rejects_sizes_beyond_its_scratch(lib):
    from paper_2606_18073_gb300 import _lib as L
    n = 65536
    nnz = (SCRATCH_BYTES - 4 * (n + 1)) // 8 + 1024     # FP32 values: 8 bytes per entry
    assert _scratch_need(n, nnz, 4) > SCRATCH_BYTES
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")   # never read: the size check comes first
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.sgks_csr_transpose_noalloc(1000, n, nnz, _p(dummy), _p(dummy), _p(dummy), L.SGKS_F32, _p(dummy),
                                        _p(dummy), _p(dummy), C.c_void_p(st))
    assert rc == L.SGKS_ERR_INVALID
    assert b"fixed scratch" in lib.sgks_last_error(None)
