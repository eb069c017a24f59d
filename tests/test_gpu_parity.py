"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Iterates x_k are compared in relative 2-norm.  The bar is 1e-10 for the FP64 form and 1e-4
for the FP32 form, raised where the method's own sensitivity makes that impossible: sGKS
never re-orthogonalises its basis, so rounding-level differences between two correct
implementations grow from iteration to iteration.  The floor of iteration k is measured with
the oracle alone: the oracle against itself with the initial basis, every gradient, every
sketched column entering the QR update, the inputs of every projected solve and every
refinement residual perturbed by (1 + u N(0,1)) -- the backward errors of those steps -- u the
unit roundoff a form uses for each step (tests/golden/make_floors.py: 2^-53 throughout for FP64;
float-float 2^-48 with an FP64 small phase; the FP32 form 2^-24 for its basis columns and
compensated sums elsewhere; FP32 sums 2^-24 throughout), the largest deviation over five seeds.
An iterate passes when its error is below max(tolerance, FACTOR * floor_k).  The FP32 form
("fp32": FP32 basis, compensated sums) is gated at every iteration; the FP32-accumulation
kernels ("fp32plain") drift from the FP64 iterates by design and are gated only while their
floor is below 1e-6.  Sparse-sign indices, CSR transposes and
integer state are compared bit-exactly."""
import json
import os
import sys

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
import parity_log
from workloads import make_problem, small_problem

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_floors import EPS, floor_curve  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4
FACTOR64 = 10.0
FACTOR32 = 10.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def check_iterates(xs, ref_xs, floor, tol, factor, name=None):
    errs = [rel(a, b) for a, b in zip(xs, ref_xs)]
    if name is None:
        name = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    parity_log.record(name, errs, floor, tol, factor)
    bad = [(k, e, floor[k]) for k, e in enumerate(errs) if e > max(tol, factor * floor[k])]
    assert not bad, f"iterates above max(tol, {factor} x floor): {bad[:5]} ... errors {errs[-3:]}"
    return errs


def load_floor(name, form):
    path = os.path.join(GOLDEN, f"floor_{name}_{form}.json")
    if not os.path.exists(path):
        pytest.skip(f"missing {path}: run tests/golden/make_floors.py")
    with open(path) as f:
        return json.load(f)["floor"]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_18073_gb300 as G
    G.build()
    return G


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_iterates(G, P, iters, precision=None, **over):
    kw = G.device_inputs(P, precision)
    kw.update(over)
    kw["max_iters"] = max(kw["max_iters"], iters)
    S = G.Solver(**kw)
    xs = [S.x().double().cpu().numpy()]
    for _ in range(iters):
        S.step()
        xs.append(S.x().double().cpu().numpy())
    return S, xs


# ------------------------------------------------------------------------ building blocks

@pytest.mark.parametrize("seed,stream,h,s,zeta", [(0, 0, 1000, 400, 8), (0, 1, 70001, 600, 8), (7, 0, 513, 9, 9),
                                                  (123456789, 1, 4097, 2048, 16), (3, 0, 333, 17, 1)])
def test_sparse_sign_indices_bit_exact(G, seed, stream, h, s, zeta):
    rows, neg = G.sparse_sign_rows(seed, stream, h, s, zeta)
    r_ref, s_ref = O.sparse_sign_rows(seed, stream, h, s, zeta)
    assert np.array_equal(rows.cpu().numpy().astype(np.int64), r_ref)
    assert np.array_equal(neg.cpu().numpy().astype(bool), s_ref < 0)


def test_csr_transpose_bit_exact(G):
    P = small_problem("ct2d")
    A = G.device_inputs(P, "fp64", transpose=True)["A"]
    M = sp.csr_matrix((P.A.val, P.A.col, P.A.row_ptr), shape=(P.m, P.n)).tocsc()
    M.sort_indices()
    assert np.array_equal(A.t_row_ptr.cpu().numpy(), M.indptr)
    assert np.array_equal(A.t_col.cpu().numpy(), M.indices)
    assert np.array_equal(A.t_val.cpu().numpy(), M.data)


@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_operators_match_oracle(G, kind, precision):
    P = small_problem(kind)
    S = G.Solver(**G.device_inputs(P, precision))
    Aop, Lop = O.make_operators(P)
    dt = S.dtype
    tol = 1e-13 if precision == "fp64" else 2e-6
    rng = np.random.default_rng(1)
    cases = [(G._lib.SGKS_APPLY_A, P.n, Aop.apply), (G._lib.SGKS_APPLY_AT, P.m, Aop.adjoint),
             (G._lib.SGKS_APPLY_L, P.n, Lop.apply), (G._lib.SGKS_APPLY_LT, P.p, Lop.adjoint),
             (G._lib.SGKS_APPLY_LTL, P.n, lambda v: Lop.adjoint(Lop.apply(v)))]
    for which, nin, ref in cases:
        v = rng.standard_normal(nin)
        if precision == "fp32":
            v = v.astype(np.float32).astype(np.float64)
        want = ref(v)
        out = torch.empty(len(want), dtype=dt, device="cuda")
        S.apply(which, torch.from_numpy(v).to("cuda", dt), out)
        assert rel(out.cpu().numpy(), want) < tol, which
    if P.sketch.kind == "sparse_sign":
        for which, h, stream in ((G._lib.SGKS_APPLY_SA, P.m, 0), (G._lib.SGKS_APPLY_SL, P.p, 1)):
            v = rng.standard_normal(h).astype(np.float32).astype(np.float64)
            want = O.sketch_operator(P.sketch, stream, h) @ v
            out = torch.empty(P.sketch.s, dtype=torch.float64, device="cuda")
            S.apply(which, torch.from_numpy(v).to("cuda", dt), out)
            assert rel(out.cpu().numpy(), want) < (1e-13 if precision == "fp64" else 2e-6)
    S.close()


def test_setup_state_matches_oracle(G):
    """W_0, S_A b and the sketched QR factors of W_0 (eq. updqr) after sgks_create."""
    P = small_problem("deblur2d", precision="fp64", n_refine=0)
    S = G.Solver(**G.device_inputs(P, "fp64"))
    ref = O.sgks(P, iters=0, record_state=True)
    d = 3
    W = S.buffer(G._lib.SGKS_BUF_W, d * P.n).cpu().numpy().reshape(d, P.n).T
    assert rel(W, ref["W"]) < 1e-13
    assert rel(S.buffer(G._lib.SGKS_BUF_SB, P.sketch.s).cpu().numpy(), ref["Sb"]) < 1e-14
    for buf, key, rows in ((G._lib.SGKS_BUF_QA, "QA", P.sketch.s), (G._lib.SGKS_BUF_QL, "QL", P.sketch.s)):
        Q = S.buffer(buf, d * rows).cpu().numpy().reshape(d, rows).T
        assert rel(Q, ref[key]) < 1e-12
    dm = P.iters + 3
    RA = S.buffer(G._lib.SGKS_BUF_RA, d * dm).cpu().numpy().reshape(d, dm).T[:d]
    assert rel(np.triu(RA), ref["RA"]) < 1e-12
    assert rel(S.buffer(G._lib.SGKS_BUF_DA, d).cpu().numpy(), ref["dA"]) < 1e-12
    S.close()


# --------------------------------------------------------------------------- iterates

@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_fp64_iterates_match_oracle(G, kind):
    P = small_problem(kind, precision="fp64") if kind in ("deblur2d", "seismic2d", "ct2d") else small_problem(kind)
    P.precision = "fp64"
    iters = P.iters
    ref = O.sgks(P, iters=iters, record_x=True)
    S, xs = gpu_iterates(G, P, iters, "fp64")
    check_iterates(xs, ref["xs"], floor_curve(P, iters, EPS["fp64"])[0], TOL64, FACTOR64)
    S.close()
    S, xs = gpu_iterates(G, P, iters, "fp64", flags=G._lib.SGKS_FLAG_GLOBAL_SMALL)
    check_iterates(xs, ref["xs"], floor_curve(P, iters, EPS["fp64"])[0], TOL64, FACTOR64)
    S.close()


def test_fp64_iterates_cgs1_and_gaussian(G):
    P = small_problem("deconv1d")                       # Gaussian sketch
    ref = O.sgks(P, iters=P.iters, record_x=True, cgs_passes=1)
    S, xs = gpu_iterates(G, P, P.iters, "fp64", cgs_passes=1)
    fl = floor_curve_cgs1(P)
    check_iterates(xs, ref["xs"], fl, TOL64, FACTOR64)
    S.close()


def floor_curve_cgs1(P):
    """Floor of the single-projection variant (oracle with cgs_passes = 1 on every run)."""
    return floor_curve(P, P.iters, EPS["fp64"], cgs_passes=1)[0]


@pytest.mark.parametrize("kind", ["deblur2d", "dynct"])
def test_fp32plain_refined_iterates_track_oracle_early(G, kind):
    """The FP32-accumulation kernels track the FP64 oracle to 1e-4 while the method's FP32-level
    floor is below 1e-6; later their iterates drift (FP32 rounding of the stored A W columns and
    FP32 cancellation in e and the gradient), with the reconstruction quality of the oracle."""
    P = small_problem(kind)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, "fp32plain")
    fl = floor_curve(P, P.iters, EPS["fp32"])[0]
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    early = [k for k in range(len(errs)) if max(fl[:k + 1]) < 1e-6]
    assert early and max(errs[k] for k in early) < TOL32, errs
    rre = rel(xs[-1], P.x_true)
    assert abs(rre - ref["rre"][-1]) < 0.05 * ref["rre"][-1]
    S.close()


@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_fp32_iterates_match_oracle(G, kind):
    """The FP32 form (FP32 basis, compensated sums, FP64 small phase and refinement solve, the
    problem's refinement steps): every iterate within max(1e-4, F x floor) of the FP64 oracle."""
    P = small_problem(kind)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, "fp32")
    check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp32"])[0], TOL32, FACTOR32)
    S.close()


def test_fp32x_is_the_fp32_form(G):
    """SGKS_PREC_FP32X names the same form as SGKS_PREC_FP32: bit-identical iterates."""
    P = small_problem("deblur2d")
    xs = []
    for prec in ("fp32", "fp32x"):
        S = G.Solver(**G.device_inputs(P, prec))
        S.solve(P.iters)
        xs.append(S.x().cpu().numpy())
        S.close()
    assert np.array_equal(xs[0], xs[1])


def asymmetric_psf(k, seed):
    """A k x k psf with no symmetry, so that a transposed or unrotated kernel shows in the iterates."""
    rng = np.random.default_rng(seed)
    h = rng.random((k, k)) + np.linspace(0.0, 1.0, k * k).reshape(k, k)
    return (h / h.sum()).astype(np.float32)


@pytest.mark.parametrize("k,nx,ny", [(3, 24, 20), (5, 100, 12), (9, 36, 24), (11, 24, 20), (9, 30, 18)])
def test_conv_rows_asymmetric_psf(G, k, nx, ny):
    """Iterates of the deblurring problem with an asymmetric psf, FP64 with one refinement step
    (gradient append, apply and fused refinement gradient all run), through the generic
    convolution rows (any psf side, any image width)."""
    P = small_problem("deblur2d", nx=nx, ny=ny, psf=asymmetric_psf(k, k), iters=12, precision="fp64",
                      n_refine=1)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, "fp64")
    check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp64"])[0], TOL64, FACTOR64)
    S.close()


def check_fp32_early(P, xs, ref):
    """FP32 iterates within TOL32 of the FP64 oracle while the plain-FP32 floor is below 1e-6."""
    fl = floor_curve(P, P.iters, EPS["fp32plain"])[0]
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    early = [i for i in range(len(errs)) if max(fl[:i + 1]) < 1e-6]
    assert early and max(errs[i] for i in early) < TOL32, errs


@pytest.mark.parametrize("k,nx,ny", [(3, 24, 20), (5, 100, 12), (7, 28, 16), (9, 40, 28), (11, 24, 20),
                                     (9, 30, 18)])
def test_conv_rows_asymmetric_psf_fp32(G, k, nx, ny):
    """The FP32 form with an asymmetric psf and two refinement steps: square sides 3 to 9 on images
    of width % 4 == 0 take the register-blocked rows (A^T as correlation, A with the rotated
    taps); side 11 and width 30 the generic rows."""
    P = small_problem("deblur2d", nx=nx, ny=ny, psf=asymmetric_psf(k, k + 1), iters=10, precision="fp32",
                      n_refine=2)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, "fp32plain")
    check_fp32_early(P, xs, ref)
    S.close()
    S, xs = gpu_iterates(G, P, P.iters, "fp32")
    check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp32"])[0], TOL32, FACTOR32)
    S.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_conv_rows_many_tiles(G, precision):
    """A 256 x 400 image (102,400 rows): the refinement gradient's CTAs take several 256-row tiles
    and the append / apply kernels many 512-row tiles; asymmetric 9 x 9 psf."""
    P = small_problem("deblur2d", nx=256, ny=400, psf=asymmetric_psf(9, 3), iters=6, s=120, precision=precision,
                      n_refine=1)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, precision)
    if precision == "fp64":
        check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp64"])[0], TOL64, FACTOR64)
    else:
        check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp32"])[0], TOL32, FACTOR32)
    S.close()


def random_csr_problem(avg_row, seed=0, n_side=24, m=700):
    """The small CT problem with A replaced by a random sparse m x n matrix of about `avg_row`
    entries per row (non-negative, like path lengths), b = A x_true + 1% noise."""
    from workloads.configs import _noisy
    from workloads.problem import OperatorDesc
    P = small_problem("ct2d", N=n_side, iters=12, precision="fp64", n_refine=0)
    rng = np.random.default_rng(seed)
    n = P.n
    rows, cols = [], []
    for i in range(m):
        k = max(1, int(rng.poisson(avg_row)))
        cols.append(np.sort(rng.choice(n, size=min(k, n), replace=False)))
        rows.append(len(cols[-1]))
    rp = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32)
    val = rng.uniform(0.1, 1.0, size=len(col)).astype(np.float32)
    P.A = OperatorDesc("csr", m, n, row_ptr=rp, col=col, val=val, nx=n_side, ny=n_side)
    P.b = _noisy(P.A, P.x_true, 0.01, np.random.default_rng(seed + 1))
    return P


@pytest.mark.parametrize("avg_row", [5, 24, 60, 160])
def test_csr_lanes_per_row(G, avg_row):
    """CSR rows of about 5, 24, 60 and 160 entries (4, 8, 16 and 32 lanes per row for A; the
    transposed rows are shorter), FP64 iterates against the oracle."""
    P = random_csr_problem(avg_row, seed=avg_row)
    ref = O.sgks(P, record_x=True)
    S, xs = gpu_iterates(G, P, P.iters, "fp64")
    check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp64"])[0], TOL64, FACTOR64)
    S.close()


@pytest.mark.parametrize("precision", ["fp32plain", "fp32", "fp64"])
def test_csr_adjoint_paths(G, precision):
    """A^T rows of ~146 entries (random 700 x 576 CSR, ~120 entries per row of A), read from the
    CSR transpose with 32 lanes per row (the interleaved slices serve operators with n >= 155,648:
    the full-size CT and dynamic-CT tests).  Against the oracle: the apply, and the iterates of a
    solve with one refinement step (the append and the refinement gradients)."""
    P = random_csr_problem(120, seed=3)
    P.n_refine = 1
    assert len(P.A.col) >= 96 * P.n
    Aop, _ = O.make_operators(P)
    S, xs = gpu_iterates(G, P, P.iters, precision)
    v = np.random.default_rng(2).standard_normal(P.m)
    if precision != "fp64":
        v = v.astype(np.float32).astype(np.float64)
    out = torch.empty(P.n, dtype=S.dtype, device="cuda")
    S.apply(G._lib.SGKS_APPLY_AT, torch.from_numpy(v).to("cuda", S.dtype), out)
    assert rel(out.cpu().numpy(), Aop.adjoint(v)) < (1e-13 if precision == "fp64" else 2e-6)
    ref = O.sgks(P, record_x=True)
    if precision == "fp64":
        check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp64"])[0], TOL64, FACTOR64)
    elif precision == "fp32":
        check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp32"])[0], TOL32, FACTOR32)
    else:
        check_fp32_early(P, xs, ref)
    S.close()


def test_programmatic_launch_changes_nothing(G, tmp_path):
    """The iteration's kernels launch with programmatic dependent launch; SGKS_PDL=0 launches them
    plainly.  Only the scheduling differs, so the solve is bit-identical (checked in a child
    process, since the switch is read once per process)."""
    import subprocess
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r)\n"
        "import paper_2606_18073_gb300 as G\n"
        "from workloads import small_problem\n"
        "G.build()\n"
        "P = small_problem('deblur2d')\n"
        "S = G.Solver(**G.device_inputs(P, 'fp32plain'))\n"
        "S.solve(P.iters)\n"
        "np.save(%r, S.x().cpu().numpy())\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), str(tmp_path / "x.npy"))
    env = dict(os.environ, SGKS_PDL="0")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    P = small_problem("deblur2d")
    S = G.Solver(**G.device_inputs(P, "fp32plain"))
    S.solve(P.iters)
    assert np.array_equal(S.x().cpu().numpy(), np.load(tmp_path / "x.npy"))
    S.close()


def test_ragged_sizes_and_extreme_sketch(G):
    """n not a multiple of the 32-row slab or 256-row tile; zeta = 1 and zeta = s."""
    for nx, ny, s, zeta in ((37, 23, 64, 1), (19, 41, 40, 16), (33, 7, 30, 8)):
        P = small_problem("deblur2d", nx=nx, ny=ny, s=s, zeta=zeta, iters=15, precision="fp64", n_refine=1)
        ref = O.sgks(P, record_x=True)
        S, xs = gpu_iterates(G, P, P.iters, "fp64")
        check_iterates(xs, ref["xs"], floor_curve(P, P.iters, EPS["fp64"])[0], TOL64, FACTOR64)
        S.close()


def test_solve_graph_replay_equals_steps_and_is_deterministic(G):
    P = small_problem("ct2d", iters=15)
    kw = G.device_inputs(P, "fp64")
    S1 = G.Solver(**kw)
    for _ in range(15):
        S1.step()
    x1 = S1.x().cpu().numpy()
    S2 = G.Solver(**kw)
    out = S2.solve(15, history=True)
    x2 = S2.x().cpu().numpy()
    assert np.array_equal(x1, x2)
    assert out["iters_done"] == 15 and out["d"] == 18 and len(out["rc"]) == 15
    ref = O.sgks(P, iters=15)
    assert np.allclose(out["rc"], ref["rc"], rtol=1e-8, atol=0)
    assert np.allclose(out["rre"], ref["rre"][1:], rtol=1e-9, atol=0)
    S3 = G.Solver(**kw)
    S3.solve(15)
    assert np.array_equal(S3.x().cpu().numpy(), x2)
    # reset with a new right-hand side equals a fresh solver on that b
    P2 = small_problem("ct2d", seed=5, iters=15)
    b2 = torch.from_numpy(P2.b).cuda()
    S3.reset(b2)
    S3.solve(15)
    kw2 = dict(kw)
    kw2["b"] = b2
    S4 = G.Solver(**kw2)
    S4.solve(15)
    assert np.array_equal(S3.x().cpu().numpy(), S4.x().cpu().numpy())
    for s in (S1, S2, S3, S4):
        s.close()


@pytest.mark.parametrize("precision", ["fp32plain", "fp32"])
def test_profile_graph_matches_steps(G, precision):
    """sgks_profile_graph runs the same kernels as sgks_step (the iterate is bit-identical) and
    counts the same launches per class as the eager profile."""
    P = small_problem("deblur2d")
    kw = G.device_inputs(P, precision)
    S1 = G.Solver(**kw)
    pe = S1.profile(6)
    S2 = G.Solver(**kw)
    pg = S2.profile(6, graph=True)
    S3 = G.Solver(**kw)
    for _ in range(6):
        S3.step()
    assert np.array_equal(S2.x().cpu().numpy(), S3.x().cpu().numpy())
    assert np.array_equal(S1.x().cpu().numpy(), S3.x().cpu().numpy())
    for k in pe:
        assert pe[k]["launches"] == pg[k]["launches"] and pe[k]["dsum"] == pg[k]["dsum"], k
        assert (pg[k]["ms"] > 0) == (pg[k]["launches"] > 0), k
    with pytest.raises(G._lib.SGKSError):
        S2.profile(10 ** 6, graph=True)
    for S in (S1, S2, S3):
        S.close()


def test_time_class_leaves_state(G):
    """sgks_time_class relaunches streaming kernels in place: the iteration that follows is the
    same, bit for bit, as without the timing; other classes and the compensated FP32 form are
    rejected."""
    P = small_problem("deblur2d")
    kw = G.device_inputs(P, "fp32plain")
    S1, S2 = G.Solver(**kw), G.Solver(**kw)
    for _ in range(4):
        S1.step()
        S2.step()
    for k in ("gradient_append", "sketch_column", "combine_refine", "gradient_refine"):
        assert S1.time_class(k, 5) > 0.0
    for _ in range(3):
        S1.step()
        S2.step()
    assert np.array_equal(S1.x().cpu().numpy(), S2.x().cpu().numpy())
    with pytest.raises(G._lib.SGKSError) as ei:
        S1.time_class("qr_append", 5)
    assert ei.value.code == G._lib.SGKS_ERR_INVALID
    S3 = G.Solver(**G.device_inputs(P, "fp32x"))
    with pytest.raises(G._lib.SGKSError) as ei:
        S3.time_class("gradient_refine", 5)
    assert ei.value.code == G._lib.SGKS_ERR_INVALID
    for S in (S1, S2, S3):
        S.close()


def test_rc_tolerance_stops(G):
    P = small_problem("deblur2d", precision="fp64", n_refine=0, iters=40)
    S = G.Solver(**G.device_inputs(P, "fp64"))
    ref = O.sgks(P, tol=1e-3)
    out = S.solve(40, tol=1e-3)
    assert out["status"] == G._lib.SGKS_STOPPED
    assert out["iters_done"] == ref["iters"]
    assert rel(S.x().cpu().numpy(), ref["x"]) < TOL64
    S.close()


def test_basis_full_is_an_error(G):
    P = small_problem("deconv1d", iters=4)
    S = G.Solver(**G.device_inputs(P, "fp64"))
    S.solve(4)
    with pytest.raises(G._lib.SGKSError) as ei:
        S.step()
    assert ei.value.code == G._lib.SGKS_ERR_STATE
    S.close()


def test_breakdown_when_basis_spans_space(G):
    """Tiny n: once W spans R^n the next gradient is (numerically) in its span."""
    P = small_problem("deconv1d", n=6, s=40, iters=30, lam=1e-1)
    S = G.Solver(**G.device_inputs(P, "fp64"))
    out = S.solve(30)
    assert out["status"] == G._lib.SGKS_BREAKDOWN
    assert out["d"] <= 6 + 1
    Aop, Lop = O.make_operators(P)
    SA, SL = O.sketch_operator(P.sketch, 0, P.m), O.sketch_operator(P.sketch, 1, P.p)
    xs = O.direct_solve(Aop, Lop, P.b, P.lam, SA, SL)
    assert rel(S.x().cpu().numpy(), xs) < 1e-8
    S.close()


def test_invalid_arguments(G):
    P = small_problem("deblur2d", precision="fp64")
    kw = G.device_inputs(P, "fp64")
    for bad in (dict(lam=-1.0), dict(sketch_rows=5), dict(zeta=17), dict(sketch_rows=4096)):
        k = dict(kw)
        k.update(bad)
        with pytest.raises(G._lib.SGKSError) as ei:
            G.Solver(**k)
        assert ei.value.code == G._lib.SGKS_ERR_INVALID


def test_nonfinite_rhs_is_reported(G):
    P = small_problem("deblur2d", precision="fp64", n_refine=0)
    kw = G.device_inputs(P, "fp64")
    kw["b"] = kw["b"].clone()
    kw["b"][3] = float("nan")
    S = G.Solver(**kw)
    with pytest.raises(G._lib.SGKSError) as ei:
        S.solve(3)
    assert ei.value.code == G._lib.SGKS_ERR_NONFINITE
    S.close()


# ----------------------------------------------------------------------- full-size configs
# Full workload sizes and iteration counts of the five test problems, launched as bench.py launches them (sgks_solve replays of
# the captured step graph after sgks_reset); iterates are read after every replay.

def gpu_graph_iterates(G, P, precision, **over):
    kw = G.device_inputs(P, precision)
    kw.update(over)
    S = G.Solver(**kw)
    S.reset(kw["b"])
    xs = [S.x().double().cpu().numpy()]
    for _ in range(P.iters):
        S.solve(1)
        xs.append(S.x().double().cpu().numpy())
    S.close()
    return xs


@pytest.mark.slow
@pytest.mark.parametrize("name", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_full_size_fp64(G, name):
    P = make_problem(name)
    P.n_refine = 0
    ref = O.sgks(P, record_x=True)
    xs = gpu_graph_iterates(G, P, "fp64")
    errs = check_iterates(xs, ref["xs"], load_floor(name, "fp64"), TOL64, FACTOR64, name=f"full_size_fp64[{name}]")
    k_strict = max([k for k, e in enumerate(errs) if e < TOL64] + [0])
    print(f"{name}: fp64 max error {max(errs):.2e}; below 1e-10 through iteration {k_strict}")


@pytest.mark.slow
@pytest.mark.parametrize("name", ["deblur2d", "dynct"])
def test_full_size_fp32_refined(G, name):
    """The FP32 form at the full workload size with the workload's refinement steps: every
    iterate within max(1e-4, F x floor_k) of the FP64 oracle."""
    P = make_problem(name)
    ref = O.sgks(P, record_x=True)
    xs = gpu_graph_iterates(G, P, "fp32")
    fl = load_floor(name, "fp32")
    errs = check_iterates(xs, ref["xs"], fl, TOL32, FACTOR32, name=f"full_size_fp32[{name}]")
    k_strict = max([k for k, e in enumerate(errs) if e < TOL32] + [0])
    print(f"{name}: fp32 max error {max(errs):.2e}, final {errs[-1]:.2e}; below 1e-4 through iteration {k_strict}")
