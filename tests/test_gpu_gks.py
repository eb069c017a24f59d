"""GKS (Algorithm 1) on the GPU (SGKS_FLAG_GKS) against the FP64 oracle's gks().

GKS keeps an orthonormal basis, so two correct FP64 implementations agree to rounding: the
oracle against itself with rounding-level gradient perturbations differs by at most 1e-14 on
these problems, and the bar is the plain 1e-10 of the FP64 path (1e-4 for FP32)."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import small_problem

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


def gks_iterates(G, P, prec):
    kw = G.device_inputs(P, prec)
    kw["n_refine"] = 0
    S = G.Solver(**kw, method="gks")
    xs = [S.x().double().cpu().numpy()]
    for _ in range(P.iters):
        S.step()
        xs.append(S.x().double().cpu().numpy())
    return S, xs


@pytest.mark.parametrize("kind", ["deconv1d", "deblur2d", "ct2d", "seismic2d", "dynct"])
def test_gks_iterates_match_oracle_fp64(G, kind):
    P = small_problem(kind)
    P.n_refine = 0
    ref = O.gks(P, record_x=True)
    S, xs = gks_iterates(G, P, "fp64")
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    assert len(errs) == P.iters + 1 and max(errs) < 1e-10, errs
    S.close()


@pytest.mark.parametrize("kind", ["deblur2d", "seismic2d"])
def test_gks_iterates_match_oracle_fp32(G, kind):
    P = small_problem(kind)
    P.n_refine = 0
    ref = O.gks(P, record_x=True)
    S, xs = gks_iterates(G, P, "fp32")
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    assert max(errs) < 1e-4, errs
    S.close()


def test_gks_graph_replay_equals_steps(G):
    P = small_problem("ct2d", iters=12)
    P.n_refine = 0
    kw = G.device_inputs(P, "fp64")
    kw["n_refine"] = 0
    S1 = G.Solver(**kw, method="gks")
    for _ in range(12):
        S1.step()
    S2 = G.Solver(**kw, method="gks")
    out = S2.solve(12)
    assert out["iters_done"] == 12 and out["d"] == 3 + 12
    assert np.array_equal(S1.x().cpu().numpy(), S2.x().cpu().numpy())
    S1.close()
    S2.close()


def test_gks_rejects_unsupported_options(G):
    P = small_problem("seismic2d")
    kw = G.device_inputs(P, "fp64")
    for bad in (dict(n_refine=1), dict(record=True), dict(precision="ff")):
        k2 = dict(kw)
        k2["n_refine"] = 0
        k2.update(bad)
        with pytest.raises(G._lib.SGKSError) as ei:
            G.Solver(**k2, method="gks")
        assert ei.value.code == G._lib.SGKS_ERR_INVALID
