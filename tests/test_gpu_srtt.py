"""SRTT sketch (eq. sketching_trig) on the GPU: the dense S_A, S_L built on the device against
the oracle's DCT-based application, and sGKS iterates with the SRTT against the oracle."""
import json
import os
import sys

import numpy as np
import pytest
import torch

import oracle as O
from oracle.sgks_oracle import sketch_operator
from workloads import small_problem
from workloads.configs import srtt_sketch

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_floors import EPS, floor_curve  # noqa: E402

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


def srtt_problem(kind, **kw):
    P = small_problem(kind, **kw)
    P.sketch = srtt_sketch(P.sketch.s, P.m, P.p, seed=5)
    return P


@pytest.mark.parametrize("kind", ["deblur2d", "ct2d"])
def test_srtt_matrices_match_oracle(G, kind):
    P = srtt_problem(kind)
    S = G.Solver(**G.device_inputs(P, "fp64"))
    rng = np.random.default_rng(0)
    for which, h, stream in ((G._lib.SGKS_APPLY_SA, P.m, 0), (G._lib.SGKS_APPLY_SL, P.p, 1)):
        v = rng.standard_normal(h)
        out = torch.empty(P.sketch.s, dtype=torch.float64, device="cuda")
        S.apply(which, torch.from_numpy(v).cuda(), out)
        want = sketch_operator(P.sketch, stream, h) @ v
        assert rel(out.cpu().numpy(), want) < 1e-13
    S.close()


@pytest.mark.parametrize("kind", ["deblur2d", "ct2d"])
def test_srtt_iterates_match_oracle(G, kind):
    P = srtt_problem(kind, precision="fp64") if kind == "deblur2d" else srtt_problem(kind)
    P.precision = "fp64"
    ref = O.sgks(P, record_x=True)
    fl = floor_curve(P, P.iters, EPS["fp64"])[0]
    S = G.Solver(**G.device_inputs(P, "fp64"))
    xs = [S.x().cpu().numpy()]
    for _ in range(P.iters):
        S.step()
        xs.append(S.x().cpu().numpy())
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    bad = [(k, e, fl[k]) for k, e in enumerate(errs) if e > max(1e-10, 100.0 * fl[k])]
    assert not bad, bad[:4]
    S.close()


@pytest.mark.parametrize("n_refine", [0, 2])
def test_srtt_backward_matches_oracle(G, n_refine):
    """The reverse sweep with the SRTT sketch (its adjoint is the dense S^T of the device rows),
    without and with refinement steps, against the oracle's sweep, FP64, to 1e-7."""
    from oracle.sgks_adjoint import loss_and_grad
    P = srtt_problem("ct2d", iters=8)
    kw = G.device_inputs(P, "fp64")
    kw["n_refine"] = n_refine
    S = G.Solver(**kw, record=True)
    S.solve(8)
    x = S.x()
    xt = torch.from_numpy(np.asarray(P.x_true)).cuda()
    bbar, lbar = S.backward((2.0 * (x - xt)).contiguous())
    S.close()
    _, bb, lb = loss_and_grad(P, 8, n_refine=n_refine)
    assert rel(bbar.cpu().numpy(), bb) < 1e-7
    assert abs(lbar - lb) <= 1e-7 * abs(lb)


def test_srtt_rejects_missing_arrays(G):
    P = srtt_problem("deblur2d")
    kw = G.device_inputs(P, "fp64")
    kw["srtt"] = kw["srtt"][:2]
    with pytest.raises(ValueError):
        G.Solver(**kw)
