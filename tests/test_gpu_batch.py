"""Batched handle (sgks_batch_*) against the FP64 oracle, instance by instance.

Each instance of a batch is its own problem solved by Algorithm 2 with the batch's sketch seed,
so its iterates are compared with the oracle run on that problem alone, under the same
floor-based tolerance as the single-handle parity tests.  Covered: CSR, convolution and dense
operators with each regularizer; groups split into powers of two (5 = 4 + 1); ragged instances
(different frame counts) in concurrent groups; refinement; the FP32 form; graph replay against
eager steps; per-instance stopping and a non-finite instance that must not disturb the others.
"""
import os
import sys

import numpy as np
import pytest
import torch

import oracle as O
import parity_log
from workloads import small_problem
from workloads.problem import SketchDesc

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_floors import EPS, FF_SCALE, floor_curve  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-10, 1e-4
FACTOR64, FACTOR32 = 10.0, 10.0


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


def share_operators(problems, s, zeta=8, seed=0):
    """Give problems with equal operators one OperatorDesc (so the batch groups them) and the
    batch's common sketch (s, zeta, seed)."""
    firsts = []
    for P in problems:
        for Q in firsts:
            same = (Q.A.kind == P.A.kind and Q.A.m == P.A.m and Q.A.n == P.A.n and Q.L == P.L)
            if same and P.A.kind == "csr":
                same = (np.array_equal(Q.A.row_ptr, P.A.row_ptr) and np.array_equal(Q.A.col, P.A.col)
                        and np.array_equal(Q.A.val, P.A.val))
            elif same and P.A.kind == "conv2d":
                same = np.array_equal(Q.A.psf, P.A.psf)
            elif same:
                same = np.array_equal(Q.A.dense, P.A.dense)
            if same:
                P.A = Q.A
                break
        else:
            firsts.append(P)
        P.sketch = SketchDesc("sparse_sign", s, zeta, seed)
    return problems


def batch_inputs(G, problems, prec):
    dt = G.io_dtype(prec)
    ops = {}
    insts = []
    for P in problems:
        if id(P.A) not in ops:
            kw = G.device_inputs(P, prec)
            ops[id(P.A)] = (kw["A"], kw["reg"])
        A, reg = ops[id(P.A)]
        insts.append(dict(A=A, reg=reg, lam=P.lam,
                          b=torch.from_numpy(np.asarray(P.b)).to("cuda", dt),
                          x_true=torch.from_numpy(np.asarray(P.x_true)).to("cuda", dt)))
    return insts


def make_batch(G, problems, prec, **over):
    P0 = problems[0]
    kw = dict(max_iters=P0.iters, n_refine=P0.n_refine, precision=prec, zeta=P0.sketch.zeta)
    kw.update(over)
    return G.Batch(batch_inputs(G, problems, prec), P0.sketch.s, P0.sketch.seed, **kw)


def batch_iterates(G, problems, prec, iters, **over):
    Bt = make_batch(G, problems, prec, **over)
    xs = [[x.double().cpu().numpy()] for x in Bt.x()]
    for _ in range(iters):
        Bt.step()
        for i, x in enumerate(Bt.x()):
            xs[i].append(x.double().cpu().numpy())
    return Bt, xs


FORM_BAR = {  # precision -> (floor model, scale of the floor, strict bar, factor on the floor)
    "fp64": (EPS["fp64"], 1.0, TOL64, FACTOR64),
    "ff": (EPS["fp64"], FF_SCALE, TOL64, FACTOR64),   # the FP64 floor scaled by 2^-48 / 2^-53
    "fp32": (EPS["fp32"], 1.0, TOL32, FACTOR32),
}


def check_instance(xs, P, prec):
    ref = O.sgks(P, iters=len(xs) - 1, record_x=True)
    eps, scale, tol, fac = FORM_BAR[prec]
    fl = [scale * v for v in floor_curve(P, len(xs) - 1, eps)[0]]
    errs = [rel(a, b) for a, b in zip(xs, ref["xs"])]
    parity_log.record(f"batch[{prec}] {P.name}", errs, fl, tol, fac)
    bad = [(k, e, fl[k]) for k, e in enumerate(errs) if e > max(tol, fac * fl[k])]
    assert not bad, f"{P.name}: iterates above max(tol, {fac} x floor): {bad[:4]}"
    return ref


def ct_instances(count, iters=15):
    A0 = small_problem("ct2d").A
    probs = [small_problem("ct2d", instance=int(i), A=A0, iters=iters)
             for i in np.linspace(0, 63, count).astype(int)]
    return share_operators(probs, s=80)


# --------------------------------------------------------------------------------- parity

@pytest.mark.parametrize("prec", ["fp64", "ff", "fp32"])
def test_batch_ct_instances_split_into_groups_match_oracle(G, prec):
    """Five CT instances (own noise and lambda_i = 10^(-4 + 3i/63)) sharing one CSR: groups 4 + 1;
    the FP64 form and the two compensated forms."""
    probs = ct_instances(5)
    Bt, xs = batch_iterates(G, probs, prec, probs[0].iters)
    ng, grp, size = Bt.layout()
    assert ng == 2 and sorted(size) == [1, 4, 4, 4, 4]
    for P, x in zip(probs, xs):
        check_instance(x, P, prec)
    Bt.close()


@pytest.mark.parametrize("prec", ["fp64", "ff", "fp32"])
@pytest.mark.parametrize("kind", ["deblur2d", "seismic2d", "deconv1d"])
def test_batch_operator_families_match_oracle(G, kind, prec):
    """Convolution + grad2d with refinement, CSR + Laplacian, dense + fd1: four instances each."""
    if kind == "deblur2d":
        probs = [small_problem("deblur2d", seed=i, precision="fp64", n_refine=2, iters=12) for i in range(4)]
        for i, P in enumerate(probs):
            P.lam = 5e-3 * (1 + i)
    elif kind == "seismic2d":
        probs = [small_problem("seismic2d", seed=i, iters=12) for i in range(4)]
    else:
        probs = [small_problem("deconv1d", seed=i, iters=10) for i in range(4)]
    share_operators(probs, s=probs[0].sketch.s)
    assert all(P.A is probs[0].A for P in probs)
    Bt, xs = batch_iterates(G, probs, prec, probs[0].iters)
    assert Bt.layout()[0] == 1
    for P, x in zip(probs, xs):
        check_instance(x, P, prec)
    Bt.close()


@pytest.mark.parametrize("prec", ["fp64", "ff", "fp32"])
def test_batch_ragged_frames_run_as_concurrent_groups(G, prec):
    """Space-time instances with 2, 3, 4 and 4 frames: three groups on their own streams."""
    probs = [small_problem("dynct", frames=F, seed=i, iters=12) for i, F in enumerate((2, 3, 4, 4))]
    share_operators(probs, s=100)
    Bt, xs = batch_iterates(G, probs, prec, probs[0].iters)
    ng, grp, size = Bt.layout()
    assert ng == 3 and grp[2] == grp[3] and len({grp[0], grp[1], grp[2]}) == 3
    for P, x in zip(probs, xs):
        check_instance(x, P, prec)
    Bt.close()


def test_batch_fp32_form(G):
    """The FP32 form (FP32 basis, compensated sums) with two refinement steps: every iterate of
    every instance within max(1e-4, F x floor) of the oracle."""
    probs = [small_problem("deblur2d", seed=i, iters=20) for i in range(4)]
    share_operators(probs, s=80)
    Bt, xs = batch_iterates(G, probs, "fp32", probs[0].iters)
    for P, x in zip(probs, xs):
        check_instance(x, P, "fp32")
        assert abs(rel(x[-1], P.x_true) - O.sgks(P)["rre"][-1]) < 0.05 * O.sgks(P)["rre"][-1]
    Bt.close()


def test_batch_fp32plain_form(G):
    """FP32 operators and accumulation: early iterates within 1e-4 of the oracle while the
    plain-FP32 floor is below 1e-6, final RRE within 5 % (as for the single handle)."""
    probs = [small_problem("deblur2d", seed=i, iters=20) for i in range(4)]
    share_operators(probs, s=80)
    Bt, xs = batch_iterates(G, probs, "fp32plain", probs[0].iters)
    for P, x in zip(probs, xs):
        ref = O.sgks(P, record_x=True)
        fl = floor_curve(P, P.iters, EPS["fp32plain"])[0]
        errs = [rel(a, b) for a, b in zip(x, ref["xs"])]
        early = [k for k in range(len(errs)) if max(fl[:k + 1]) < 1e-6]
        assert early and max(errs[k] for k in early) < TOL32, errs
        assert abs(rel(x[-1], P.x_true) - ref["rre"][-1]) < 0.05 * ref["rre"][-1]
    Bt.close()


def test_batch_instance_equals_single_handle(G):
    """The batch changes the schedule, not the method: instance i tracks a single handle on the
    same problem to the FP64 parity bar."""
    probs = ct_instances(4, iters=12)
    Bt = make_batch(G, probs, "fp64")
    Bt.solve(12)
    xb = [x.cpu().numpy() for x in Bt.x()]
    for P, x in zip(probs, xb):
        S = G.Solver(**G.device_inputs(P, "fp64"))
        S.solve(12)
        assert rel(x, S.x().cpu().numpy()) < 1e-9
        S.close()
    Bt.close()


# ---------------------------------------------------------------------- graph and control

def test_batch_graph_replay_equals_steps(G):
    probs = ct_instances(3, iters=10)
    B1 = make_batch(G, probs, "fp64")
    for _ in range(10):
        B1.step()
    x1 = [x.cpu().numpy() for x in B1.x()]
    B2 = make_batch(G, probs, "fp64")
    out = B2.solve(10, history=True)
    x2 = [x.cpu().numpy() for x in B2.x()]
    for a, b, o in zip(x1, x2, out):
        assert np.array_equal(a, b)
        assert o["iters_done"] == 10 and len(o["rc"]) == 10
    # reset with the same right-hand sides reproduces the solve bit for bit
    B2.reset([torch.from_numpy(np.asarray(P.b)).cuda() for P in probs])
    B2.solve(10)
    for a, b in zip(x2, B2.x()):
        assert np.array_equal(a, b.cpu().numpy())
    B1.close()
    B2.close()


def test_batch_tolerance_stops_each_instance_on_its_own(G):
    # (seed, lambda) pairs whose oracle runs stop at iterations 15, 6, 31 and 22
    probs = []
    for seed, lam in ((0, 5e-3), (1, 1e-2), (0, 1e-3), (1, 2e-3)):
        P = small_problem("deblur2d", seed=seed, precision="fp64", n_refine=0, iters=40)
        P.lam = lam
        probs.append(P)
    share_operators(probs, s=80)
    Bt = make_batch(G, probs, "fp64")
    out = Bt.solve(40, tol=1e-3)
    xs = Bt.x()
    done = []
    for P, o, x in zip(probs, out, xs):
        ref = O.sgks(P, tol=1e-3)
        assert o["status"] == G._lib.SGKS_STOPPED
        assert o["iters_done"] == ref["iters"]
        fl = floor_curve(P, ref["iters"], EPS["fp64"])[0]
        assert rel(x.cpu().numpy(), ref["x"]) < max(TOL64, FACTOR64 * fl[-1])
        done.append(o["iters_done"])
    assert len(set(done)) > 1, done      # the instances really stopped at different iterations
    Bt.close()


def test_batch_nonfinite_instance_does_not_disturb_the_others(G):
    probs = ct_instances(4, iters=10)
    insts = batch_inputs(G, probs, "fp64")
    insts[1]["b"][3] = float("nan")
    Bt = G.Batch(insts, 80, 0, max_iters=10, precision="fp64")
    with pytest.raises(G._lib.SGKSError) as ei:
        Bt.solve(10)
    assert ei.value.code == G._lib.SGKS_ERR_NONFINITE
    st = Bt.status()
    assert st[1] == G._lib.SGKS_ERR_NONFINITE and st[0] == st[2] == st[3] == G._lib.SGKS_OK
    xs = Bt.x()
    for i in (0, 2, 3):
        ref = O.sgks(probs[i], iters=10)
        assert rel(xs[i].cpu().numpy(), ref["x"]) < 1e-8
    Bt.close()


def test_batch_invalid_arguments(G):
    probs = ct_instances(2, iters=5)
    insts = batch_inputs(G, probs, "fp64")
    with pytest.raises(G._lib.SGKSError) as ei:    # the float-float form exists for batches only
        G.Solver(**G.device_inputs(probs[0], "ff"))
    assert ei.value.code == G._lib.SGKS_ERR_INVALID
    insts[1]["lam"] = 0.0
    with pytest.raises(G._lib.SGKSError) as ei:
        G.Batch(insts, 80, 0, max_iters=5, precision="fp64")
    assert ei.value.code == G._lib.SGKS_ERR_INVALID and "instance 1" in str(ei.value)
    insts[1]["lam"] = 1.0
    with pytest.raises(G._lib.SGKSError) as ei:
        G.Batch(insts, 7, 0, max_iters=5, precision="fp64")      # s < ell + max_iters
    assert ei.value.code == G._lib.SGKS_ERR_INVALID


def test_batch_autotune_keeps_parity_and_caches(G):
    """SGKS_FLAG_AUTOTUNE times the tile candidates after the setup and keeps the fastest; the
    iterates still match the oracle, and a second batch of the same shape reuses the choice."""
    probs = ct_instances(4, iters=12)
    Bt, xs = batch_iterates(G, probs, "fp64", 12, autotune=True)
    cfg = Bt.config(0)
    assert cfg.startswith("slice") or cfg == "cached", cfg
    for P, x in zip(probs, xs):
        check_instance(x, P, "fp64")
    Bt.close()
    B2 = make_batch(G, probs, "fp64", autotune=True)
    assert B2.config(0) == "cached"
    B2.close()


@pytest.mark.parametrize("count,prec,tol", [(33, "fp64", 1e-10), (128, "fp64", 1e-10), (64, "fp32", 1e-4),
                                            (64, "fp32plain", 1e-4), (128, "ff", 1e-10), (3, "ff", 1e-10),
                                            (2, "fp32", 1e-4)])
def test_batch_large_groups(G, count, prec, tol):
    """Wide and narrow groups: 32 + 1 and 128 instances in FP64 (two instance passes per warp at
    128), 64 in each FP32 form, 128 and 2 + 1 in float-float, 2 in FP32; final iterate of every
    instance after 8 iterations against the oracle (at 8 iterations the method's floor is far
    below the bar)."""
    A0 = small_problem("ct2d").A
    rng = np.random.default_rng(11)
    probs = [small_problem("ct2d", instance=int(i), A=A0, iters=8) for i in rng.integers(0, 64, size=count)]
    share_operators(probs, s=80)
    Bt = make_batch(G, probs, prec)
    Bt.solve(8)
    xs = Bt.x()
    worst = max(rel(x.double().cpu().numpy(), O.sgks(P, iters=8)["x"]) for x, P in zip(xs, probs))
    assert worst < tol, worst
    Bt.close()


@pytest.mark.parametrize("prec", ["fp64", "ff"])
def test_batch_combine_timeout_stops_only_its_group(G, prec, monkeypatch):
    """The bounded waits of the bulk-copy combine: with SGKS_TEST_TIMEOUT_GROUP=0 the first group's
    ring reports a timeout at its first wait (a wait limit of zero rounds; every copy already
    issued still lands and is drained).  That group's instances stop with the timeout status,
    which the solve reports as a CUDA error; the other group's instances are unharmed."""
    probs = [small_problem("dynct", frames=F, seed=i, iters=6) for i, F in enumerate((2, 2, 3, 3))]
    share_operators(probs, s=100)
    monkeypatch.setenv("SGKS_TEST_TIMEOUT_GROUP", "0")
    Bt = make_batch(G, probs, prec)
    monkeypatch.delenv("SGKS_TEST_TIMEOUT_GROUP")
    ng, grp, _ = Bt.layout()
    assert ng == 2 and grp[0] == grp[1] == 0 and grp[2] == grp[3] == 1
    with pytest.raises(G._lib.SGKSError) as ei:
        Bt.solve(6)
    assert ei.value.code == G._lib.SGKS_ERR_CUDA
    st = Bt.status()
    assert st[0] == st[1] == G._lib.SGKS_ERR_CUDA and st[2] == st[3] == G._lib.SGKS_OK
    xs = Bt.x()
    for i in (2, 3):
        ref = O.sgks(probs[i], iters=6)
        assert rel(xs[i].double().cpu().numpy(), ref["x"]) < 1e-9
    Bt.close()
    # a batch created without the variable runs every group
    B2 = make_batch(G, probs, prec)
    B2.solve(6)
    assert all(c == G._lib.SGKS_OK for c in B2.status())
    B2.close()


# ------------------------------------------------------------------------- full-size batches
# The two batched workloads at full size, launched as bench.py launches them (one captured graph
# replayed per iteration), against the oracle run on single instances alone.  The GPU iterates are
# collected first and saved; the oracle runs afterwards in spawned processes (one per instance),
# each comparing its own iterates and returning the error curve.

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_floor(tag):
    import json
    path = os.path.join(GOLDEN, f"floor_{tag}.json")
    if not os.path.exists(path):
        pytest.skip(f"missing {path}: run tests/golden/make_floors.py")
    with open(path) as f:
        return json.load(f)["floor"]


def _oracle_errors(args):
    """Spawned worker: oracle iterates of one instance against the saved GPU iterates."""
    kind, kw, path = args
    import numpy as np
    import oracle as O
    from workloads import make_problem
    kw = dict(kw)
    sketch_seed = kw.pop("sketch_seed", None)
    P = make_problem(kind, **kw)
    if sketch_seed is not None:   # a batch shares one sketch: the seed of its first instance
        P.sketch.seed = sketch_seed
    if kind == "ct2d":
        P.n_refine = 0
    ref = O.sgks(P, record_x=True)
    xs = np.load(path)
    return [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(xs, ref["xs"])]


def _compare_in_workers(cases):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(cases)) as pool:
        return pool.map(_oracle_errors, cases)


def _graph_iterates(Bt, iters, which):
    xs = {i: [] for i in which}
    for k in range(iters + 1):
        if k:
            Bt.solve(1)
        for i, x in enumerate(Bt.x(which)):
            if x is not None:
                xs[i].append(x.double().cpu().numpy())
    return {i: np.stack(v) for i, v in xs.items()}


@pytest.mark.slow
def test_full_size_ct_batch_ff(G, tmp_path):
    """512^2 CT, 64 right-hand sides x lambda_i, 150 iterations, float-float form (the bench's
    headline workload): instances 0, 21, 42 and 63 against the oracle at every iteration,
    max(1e-10, 10 x floor_k), floor_k the instance's FP64 floor scaled by 2^-48 / 2^-53."""
    from workloads.configs import ct_op, make_ct2d
    A0 = ct_op(512, np.arange(180) * 1.0, 725)
    probs = [make_ct2d(instance=i, A=A0, precision="ff") for i in range(64)]
    Bt = make_batch(G, probs, "ff", autotune=True)
    which = (0, 21, 42, 63)
    xs = _graph_iterates(Bt, 150, which)
    Bt.close()
    cases = []
    for i in which:
        path = str(tmp_path / f"x{i}.npy")
        np.save(path, xs[i])
        cases.append(("ct2d", {"instance": i, "A": A0}, path))
    del xs
    errs = _compare_in_workers(cases)
    for i, e in zip(which, errs):
        fl = [FF_SCALE * v for v in _load_floor("ct2d_fp64" if i == 42 else f"ct2d_instance{i}_fp64")]
        parity_log.record(f"full_size_ct_batch_ff[{i}]", e, fl, TOL64, FACTOR64)
        bad = [(k, v, fl[k]) for k, v in enumerate(e) if v > max(TOL64, FACTOR64 * fl[k])]
        assert not bad, f"instance {i}: {bad[:4]}"


@pytest.mark.slow
def test_full_size_dynct_batch_fp32(G, tmp_path):
    """Dynamic CT, 16 ragged instances (frames 8, 16, 24, 32; seeds 0..15), 200 iterations with 3
    refinement steps, FP32 form: one instance per frame count (seeds 0..3) against the oracle at
    every iteration, max(1e-4, 10 x floor_k) with the instance's FP32 floor.  The batch shares one
    sketch (the seed of instance 0), so the oracle and the floors use sketch seed 0 throughout."""
    from workloads.configs import dynct_frame_ops, make_dynct
    ops = dynct_frame_ops(128, 32)
    frames = [8, 16, 24, 32] * 4
    probs, shared = [], {}
    for i, F in enumerate(frames):
        P = make_dynct(seed=i, frames=F, frame_ops=ops)
        P.A = shared.setdefault(F, P.A)
        probs.append(P)
    Bt = make_batch(G, probs, "fp32", autotune=True)
    assert Bt.layout()[0] == 4
    which = (0, 1, 2, 3)
    xs = _graph_iterates(Bt, 200, which)
    Bt.close()
    cases = []
    for i in which:
        path = str(tmp_path / f"x{i}.npy")
        np.save(path, xs[i])
        cases.append(("dynct", {"seed": i, "frames": frames[i], "sketch_seed": probs[0].sketch.seed}, path))
    del xs
    errs = _compare_in_workers(cases)
    for i, e in zip(which, errs):
        fl = _load_floor(f"dynct_seed{i}_frames{frames[i]}_sketch_seed0_fp32" if i else "dynct_seed0_frames8_fp32")
        parity_log.record(f"full_size_dynct_batch_fp32[{i}]", e, fl, TOL32, FACTOR32)
        bad = [(k, v, fl[k]) for k, v in enumerate(e) if v > max(TOL32, FACTOR32 * fl[k])]
        assert not bad, f"instance {i} ({frames[i]} frames): {bad[:4]}"


@pytest.mark.parametrize("prec", ["ff", "fp32"])
def test_batch_tiled_and_row_forward_passes_agree(G, prec):
    """A w through pixel tiles (partials per ray and tile, summed in entry order) and through the
    CSR-row kernel (SGKS_FLAG_NO_TILES): both match the oracle, on CT instances and on the
    space-time operator of two frames (tiles per frame), and the tiled solve is reproducible."""
    probs = ct_instances(4, iters=12) + []
    Bt, xs = batch_iterates(G, probs, prec, probs[0].iters)
    Bt.close()
    Bn, xn = batch_iterates(G, probs, prec, probs[0].iters, tiles=False)
    Bn.close()
    for P, a, b in zip(probs, xs, xn):
        check_instance(a, P, prec)
        check_instance(b, P, prec)
    B2, x2 = batch_iterates(G, probs, prec, probs[0].iters)
    B2.close()
    for a, b in zip(xs, x2):
        assert np.array_equal(a[-1], b[-1])
    dyn = [small_problem("dynct", frames=2, seed=i, iters=10) for i in range(2)]
    share_operators(dyn, s=100)
    Bd, xd = batch_iterates(G, dyn, prec, dyn[0].iters)
    Bd.close()
    for P, a in zip(dyn, xd):
        check_instance(a, P, prec)
