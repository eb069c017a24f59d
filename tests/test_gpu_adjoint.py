"""Differentiable form: sgks_backward against the FP64 oracle's reverse sweep and against
central finite differences of the GPU forward map; the torch autograd Function on top.

Loss l = ||x_K - x_true||^2 after K iterations, without refinement or with n_refine q = 0
refinement steps per iteration (Sec. 3.1).  In FP64 the GPU derivative tracks the oracle's to
1e-7 (both are exact derivatives of forward maps that agree to the method's rounding floor);
the FP32 form is compared loosely.
"""
import numpy as np
import pytest
import torch

from oracle.sgks_adjoint import loss_and_grad
from workloads import make_problem, small_problem

pytestmark = pytest.mark.gpu


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


def gpu_loss_grad(G, S, P, b, iters):
    S.reset(b)
    S.solve(iters)
    x = S.x()
    xt = torch.from_numpy(np.asarray(P.x_true)).to(x.device, x.dtype)
    loss = float(torch.sum((x.double() - xt.double()) ** 2))
    bbar, lbar = S.backward((2.0 * (x - xt)).contiguous())
    return loss, bbar.double().cpu().numpy(), lbar


def recording_solver(G, P, prec, n_refine=0):
    kw = G.device_inputs(P, prec)
    kw["n_refine"] = n_refine
    return G.Solver(**kw, record=True), kw["b"]


@pytest.mark.parametrize("kind,iters", [("seismic2d", 12), ("deblur2d", 10), ("ct2d", 10), ("deconv1d", 8),
                                        ("dynct", 8)])
def test_backward_matches_oracle_fp64(G, kind, iters):
    P = small_problem(kind, iters=iters)
    P.n_refine = 0
    S, b = recording_solver(G, P, "fp64")
    loss, bbar, lbar = gpu_loss_grad(G, S, P, b, iters)
    L0, bb, lb = loss_and_grad(P, iters)
    assert abs(loss - L0) <= 1e-9 * L0
    assert rel(bbar, bb) < 1e-7
    assert abs(lbar - lb) <= 1e-7 * abs(lb)
    # the call leaves the forward state as it was: a second call (captured into a graph) and a
    # third (a replay of it) give the same numbers; a replay with 2 xbar gives exactly twice them
    # (scaling by 2 commutes with every rounding), so the graph reads the new xbar
    xt = torch.from_numpy(np.asarray(P.x_true)).cuda()
    xbar = (2.0 * (S.x() - xt)).contiguous()
    b2, l2 = S.backward(xbar)
    assert np.array_equal(b2.cpu().numpy(), bbar) and l2 == lbar
    b3, l3 = S.backward(xbar)
    assert np.array_equal(b3.cpu().numpy(), bbar) and l3 == lbar
    b4, l4 = S.backward((2.0 * xbar).contiguous())
    assert np.array_equal(b4.cpu().numpy(), 2.0 * bbar) and l4 == 2.0 * lbar
    # a new solve with the same K: the replayed graph reads the new forward state
    S.reset(b)
    S.solve(iters)
    b5, l5 = S.backward(xbar)
    assert np.array_equal(b5.cpu().numpy(), bbar) and l5 == lbar
    S.close()


def test_backward_matches_gpu_finite_differences(G):
    P = small_problem("seismic2d", iters=12)
    P.n_refine = 0
    S, b = recording_solver(G, P, "fp64")
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, 12)
    h = 1e-6
    lam0 = P.lam

    def loss_at(bv, lam):
        S.set_lambda(lam)
        S.reset(bv)
        S.solve(12)
        x = S.x().cpu().numpy()
        return float(np.sum((x - np.asarray(P.x_true)) ** 2))

    fd = (loss_at(b, lam0 + h) - loss_at(b, lam0 - h)) / (2 * h)
    assert abs(lbar - fd) <= 1e-6 * abs(fd)
    rng = np.random.default_rng(5)
    for _ in range(3):
        dv = torch.from_numpy(rng.standard_normal(P.m)).cuda()
        fd = (loss_at(b + h * dv, lam0) - loss_at(b - h * dv, lam0)) / (2 * h)
        an = float(bbar @ dv.cpu().numpy())
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-10
    S.close()


@pytest.mark.parametrize("kind,iters,n_refine", [("seismic2d", 12, 1), ("deblur2d", 10, 2), ("ct2d", 8, 1),
                                                  ("deconv1d", 8, 3), ("dynct", 8, 2)])
def test_backward_with_refinement_matches_oracle(G, kind, iters, n_refine):
    """Held to 1e-7, or to 10 x the oracle's own rounding floor where that is larger: the terms
    of a refinement step carry y^{r-1} - y^r, a difference at the rounding level once the steps
    have converged (on the 1-D deconvolution with 3 steps the oracle against itself, with
    rounding-level perturbations of its gradient columns, differs by ~1e-7 in dl/dlambda)."""
    P = small_problem(kind, iters=iters)
    S, b = recording_solver(G, P, "fp64", n_refine)
    loss, bbar, lbar = gpu_loss_grad(G, S, P, b, iters)
    L0, bb, lb = loss_and_grad(P, iters, n_refine=n_refine)
    _, _, fb, fl = adjoint_floor(P, iters, n_refine=n_refine)
    assert abs(loss - L0) <= 1e-9 * L0
    assert rel(bbar, bb) < max(1e-7, 10.0 * fb)
    assert abs(lbar - lb) <= max(1e-7, 10.0 * fl) * abs(lb)
    xt = torch.from_numpy(np.asarray(P.x_true)).cuda()
    xbar = (2.0 * (S.x() - xt)).contiguous()
    for _ in range(2):   # captured, then replayed
        b2, l2 = S.backward(xbar)
        assert np.array_equal(b2.cpu().numpy(), bbar) and l2 == lbar
    # the refinement steps change the derivative: the one without them is measurably different
    _, bb0, _ = loss_and_grad(P, iters, n_refine=0)
    assert rel(bb0, bb) > 1e3 * rel(bbar, bb)
    S.close()


def test_backward_with_refinement_matches_gpu_finite_differences(G):
    P = small_problem("deblur2d", iters=10)
    S, b = recording_solver(G, P, "fp64", 2)
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, 10)
    h = 1e-6
    lam0 = P.lam

    def loss_at(bv, lam):
        S.set_lambda(lam)
        S.reset(bv)
        S.solve(10)
        x = S.x().cpu().numpy()
        return float(np.sum((x - np.asarray(P.x_true)) ** 2))

    fd = (loss_at(b, lam0 * (1 + h)) - loss_at(b, lam0 * (1 - h))) / (2 * h * lam0)
    assert abs(lbar - fd) <= 1e-6 * abs(fd)
    rng = np.random.default_rng(6)
    for _ in range(2):
        dv = torch.from_numpy(rng.standard_normal(P.m)).cuda()
        fd = (loss_at(b + h * dv, lam0) - loss_at(b - h * dv, lam0)) / (2 * h)
        an = float(bbar @ dv.cpu().numpy())
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-10
    S.close()


def test_autograd_function(G):
    P = small_problem("ct2d", iters=8)
    P.n_refine = 0
    S, b = recording_solver(G, P, "fp64")
    bb = b.clone().requires_grad_(True)
    lam = torch.tensor(P.lam, dtype=torch.float64, requires_grad=True)
    x = G.solve_differentiable(S, bb, lam, 8)
    xt = torch.from_numpy(np.asarray(P.x_true)).cuda()
    loss = torch.sum((x - xt) ** 2)
    gb, gl = torch.autograd.grad(loss, (bb, lam))
    L0, bref, lref = loss_and_grad(P, 8)
    assert abs(float(loss.detach()) - L0) <= 1e-9 * L0
    assert rel(gb.cpu().numpy(), bref) < 1e-7
    assert abs(float(gl) - lref) <= 1e-7 * abs(lref)
    # a new lambda through the same solver
    lam2 = torch.tensor(2.0 * P.lam, dtype=torch.float64, requires_grad=True)
    x2 = G.solve_differentiable(S, bb, lam2, 8)
    gl2 = torch.autograd.grad(torch.sum((x2 - xt) ** 2), lam2)[0]
    P.lam = 2.0 * P.lam
    assert abs(float(gl2) - loss_and_grad(P, 8)[2]) <= 1e-7 * abs(float(gl2))
    S.close()


def test_backward_fp32_form(G):
    P = small_problem("seismic2d", iters=12)
    P.n_refine = 0
    S, b = recording_solver(G, P, "fp32")
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, 12)
    _, bb, lb = loss_and_grad(P, 12)
    assert rel(bbar, bb) < 2e-2
    assert abs(lbar - lb) <= 2e-2 * abs(lb)
    S.close()


def test_backward_fp32_form_with_refinement(G):
    """The FP32 form's derivative with 2 refinement steps, against the FP64 oracle's: FP32
    operators and W, FP64 sketched QR, solves and refinement reductions, compared as loosely as
    the form without refinement."""
    P = small_problem("deblur2d", iters=10)
    S, b = recording_solver(G, P, "fp32", 2)
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, 10)
    _, bb, lb = loss_and_grad(P, 10, n_refine=2)
    print(f"fp32 refined: rel(bbar) = {rel(bbar, bb):.2e}, rel(lambdabar) = {abs(lbar - lb) / abs(lb):.2e}")
    assert rel(bbar, bb) < 2e-2
    assert abs(lbar - lb) <= 2e-2 * abs(lb)
    S.close()


def test_backward_errors(G):
    P = small_problem("seismic2d", iters=4)
    kw = G.device_inputs(P, "fp64")
    S = G.Solver(**kw)                       # not recording
    S.solve(4)
    with pytest.raises(G._lib.SGKSError) as ei:
        S.backward(torch.zeros(P.n, dtype=torch.float64, device="cuda"))
    assert ei.value.code == G._lib.SGKS_ERR_STATE
    S.close()
    with pytest.raises(G._lib.SGKSError) as ei:   # float-float is a batch form
        G.Solver(**G.device_inputs(P, "ff"), record=True)
    assert ei.value.code == G._lib.SGKS_ERR_INVALID
    S = G.Solver(**kw, record=True)
    S.solve(4)
    S.set_lambda(2.0 * P.lam)
    with pytest.raises(G._lib.SGKSError) as ei:
        S.backward(torch.zeros(P.n, dtype=torch.float64, device="cuda"))
    assert ei.value.code == G._lib.SGKS_ERR_STATE
    with pytest.raises(G._lib.SGKSError):
        S.step()
    S.close()


def adjoint_floor(P, iters, seed=0, n_refine=0):
    """Rounding floor of the reverse sweep itself: the oracle's gradient against the oracle's
    gradient with every forward gradient column perturbed by (1 + 2^-53 N(0, 1))."""
    from oracle import sgks_oracle as OS
    _, b0, l0 = loss_and_grad(P, iters, n_refine=n_refine)
    rng = np.random.default_rng(seed)
    orig = OS.gradient
    OS.gradient = lambda A, L, b, lam, x: orig(A, L, b, lam, x) * (1.0 + 2.0 ** -53 * rng.standard_normal(P.n))
    try:
        _, b1, l1 = loss_and_grad(P, iters, n_refine=n_refine)
    finally:
        OS.gradient = orig
    return b0, l0, rel(b1, b0), abs(l1 - l0) / abs(l0)


@pytest.mark.slow
@pytest.mark.parametrize("iters", [40, 80])
def test_full_size_seismic_gradient(G, iters):
    """The seismic travel-time problem (256 x 256, 8192 rays, Laplacian L, 80 iterations).  The
    derivative of the unrolled solve goes through G_j^{-1} = T_j^{-1} T_j^{-T}, i.e. the square of
    the projected problem's condition number, which grows as the non-orthogonal basis fills up:
    the FP64 oracle against itself with rounding-level perturbations differs by ~1e-2 at 80
    iterations (1e-8 at 40).  The GPU gradient is held to 10 x that floor, and dl/dlambda also to
    central differences of the GPU forward map (which needs no G^{-1})."""
    P = make_problem("seismic2d")
    P.n_refine = 0
    S, b = recording_solver(G, P, "fp64")
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, iters)
    bb, lb, fb, fl = adjoint_floor(P, iters)
    print(f"seismic {iters} its: rel(bbar) = {rel(bbar, bb):.2e} (floor {fb:.2e}), "
          f"rel(lambdabar) = {abs(lbar - lb) / abs(lb):.2e} (floor {fl:.2e})")
    assert rel(bbar, bb) <= max(1e-6, 10.0 * fb)
    assert abs(lbar - lb) <= max(1e-6, 10.0 * fl) * abs(lb)
    h = 1e-6 * P.lam
    lam0 = P.lam
    S.set_lambda(lam0 + h)
    lp = gpu_loss_grad(G, S, P, b, iters)[0]
    S.set_lambda(lam0 - h)
    lm = gpu_loss_grad(G, S, P, b, iters)[0]
    fd = (lp - lm) / (2 * h)
    print(f"dl/dlambda {lbar:.6e}, central difference {fd:.6e}")
    assert abs(lbar - fd) <= max(1e-4, 10.0 * fl) * abs(fd)
    S.close()


@pytest.mark.slow
def test_full_size_deblur_refined_gradient(G):
    """The 256 x 256 deblurring problem with its 2 refinement steps per iteration, 40 iterations,
    FP64: the sweep runs back through 80 refinement steps.  The oracle against itself under
    rounding-level perturbations differs by ~2e-7 in dl/db here (O(1) by 100 iterations, where the
    unrolled derivative carries no digits); the GPU is held to 10 x that floor."""
    P = make_problem("deblur2d")
    P.iters = 40
    S, b = recording_solver(G, P, "fp64", P.n_refine)
    _, bbar, lbar = gpu_loss_grad(G, S, P, b, 40)
    bb, lb, fb, fl = adjoint_floor(P, 40, n_refine=P.n_refine)
    print(f"deblur refined 40 its: rel(bbar) = {rel(bbar, bb):.2e} (floor {fb:.2e}), "
          f"rel(lambdabar) = {abs(lbar - lb) / abs(lb):.2e} (floor {fl:.2e})")
    assert rel(bbar, bb) <= max(1e-6, 10.0 * fb)
    assert abs(lbar - lb) <= max(1e-6, 10.0 * fl) * abs(lb)
    S.close()


@pytest.mark.parametrize("n_refine", [0, 1])
def test_backward_basis_adjoint_in_host_memory_is_bit_identical(G, n_refine):
    """SGKS_FLAG_BW_HOST keeps the reverse sweep's basis adjoint (as large as W) in pinned host
    memory that the kernels reach over the CPU-GPU link: dl/db and dl/dlambda are the same, bit
    for bit, as with the adjoint in device memory -- seismic 256^2 at K = 80 (and K = 20 with a
    refinement step), eager and replayed."""
    P = make_problem("seismic2d")
    K = 80 if n_refine == 0 else 20
    out = []
    for flags in (0, G._lib.SGKS_FLAG_BW_HOST):
        kw = G.device_inputs(P, "fp64")
        kw["n_refine"] = n_refine
        kw["max_iters"] = K
        S = G.Solver(**kw, record=True, flags=flags)
        S.solve(K)
        x = S.x()
        xt = torch.from_numpy(np.asarray(P.x_true)).to(x.device, x.dtype)
        xbar = (2.0 * (x - xt)).contiguous()
        r1 = S.backward(xbar)
        r2 = S.backward(xbar)
        r3 = S.backward(xbar)   # replayed from the captured graph
        S.close()
        for r in (r2, r3):
            assert torch.equal(r[0], r1[0]) and r[1] == r1[1]
        out.append((r1[0].cpu().numpy(), r1[1]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_backward_host_flag_needs_record(G):
    P = small_problem("seismic2d", iters=4)
    with pytest.raises(G._lib.SGKSError) as ei:
        G.Solver(**G.device_inputs(P, "fp64"), flags=G._lib.SGKS_FLAG_BW_HOST)
    assert ei.value.code == G._lib.SGKS_ERR_INVALID
