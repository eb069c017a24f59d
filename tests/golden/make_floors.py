"""Write tests/golden/floor_<config>_<form>.json: the inherent iterate-agreement floor of sGKS.

sGKS builds its basis from gradients at earlier iterates and never re-orthogonalises, so a
perturbation at the level of rounding grows from one iteration to the next.  Two correct
implementations that differ only in the order of floating-point operations therefore drift
apart.  This script measures that drift from oracle/ alone: it runs the oracle (oracle.sgks)
once, and then, once per seed, Algorithm 2 with the data flow of the GPU kernels (A w kept per
basis column, e = (A W) y - b from the same y as x = W y, the sketched column taken from the kept
A w; _perturbed_aw, built from oracle primitives) with every step that rounds given the backward
error of that step -- each term or entry multiplied by (1 + u * N(0,1)), u the unit roundoff the
form uses for it -- and records, for every k, the largest ||x_k - x'_k|| / ||x'_k|| over the
seeds (eight by default).  The deviation so includes what the two data flows differ by in
floating point: on the 32-frame dynamic CT, the GPU's FP64 iterates jump at iteration 139 while
perturbed runs in the oracle's own data flow (e = A x - b) jumped at 153 to 179 over 16 seeds;
in the kernels' data flow they jump at 152 to 159.  The steps:
  basis      the initial basis W_0 and every gradient (eq. gradient) as stored in the basis;
  sum        one rounding per term of the sums: the terms W_j y_j of x = W y (which reach
             e = A W y - b through A), the b term of the residual, the residual entering A^T,
             and the two terms A^T e and lam L^T L x of every gradient (eq. gradient), in the
             basis gradient and in every refinement residual;
  column     every sketched column entering the QR update (eq. updqr);
  solve      the inputs R_A, R_L, d_A of every projected solve (eq. projected_sketched_bis);
  refine     the refinement residual r(y) as stored.
Per term, not per output: the residual is near the noise level and the gradient tends to zero
as the iterates converge, so their rounding errors are set by their terms, not their values.

    form        basis      sum        column     solve      refine
    fp64        2^-53      2^-53      2^-53      2^-53      2^-53
    fp32        2^-24      2^-48      2^-48      2^-53      2^-48   (FP32 basis, compensated sums)
    fp32plain   2^-24      2^-24      2^-24      2^-24      2^-24   (FP32 sums everywhere)

(In EPS below, "gradient" is the basis column, and "combine" the sum x = W y.)

The float-float form has no floor of its own: it performs the FP64 form's operations with unit
roundoff 2^-48 in place of 2^-53 (its small phase is FP64), and the deviation of an iterate grows
linearly with the rounding level, so its floor is FF_SCALE = 2^5 times the FP64 floor.  (On the
512^2 CT instance 0 the GPU's float-float and FP64 batches deviate from the oracle in ratios of 10
to 55 over k = 50..150.  The per-step model with 2^-48 in the float-float steps gives floors barely
above the FP64 ones -- there the fresh 2^-53 perturbation of the projected solve dominates -- and
falls short of the measured float-float deviation by up to 40x.)

The per-seed curves are kept too.  The parity tests accept a CUDA iterate when its error against
the oracle is below max(tolerance, FACTOR * floor_k).

Only oracle/ and workloads/ are used.  Run:
    python tests/golden/make_floors.py [config[@key=value,...][:form] ...] [--seeds N] [--jobs J]
A target such as ct2d@instance=21:fp64 passes instance=21 to the workload generator and writes
floor_ct2d_instance21_fp64.json (the batched tests compare single instances of a batch).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

U53, U48, U24 = 2.0 ** -53, 2.0 ** -48, 2.0 ** -24
EPS = {  # form -> unit roundoff of each step that rounds
    "fp64": {"gradient": U53, "column": U53, "solve": U53, "refine": U53, "combine": U53, "sum": U53},
    "fp32": {"gradient": U24, "column": U48, "solve": U53, "refine": U48, "combine": U48, "sum": U48},
    "fp32plain": {"gradient": U24, "column": U24, "solve": U24, "refine": U24, "combine": U24, "sum": U24},
}
FF_SCALE = 2.0 ** 5   # float-float floor = FF_SCALE x FP64 floor (2^-48 / 2^-53)
FORMS = {  # config -> (forms, n_refine used with the FP64 and float-float forms)
    "deconv1d": (["fp64"], 0),
    "deblur2d": (["fp64", "fp32"], 0),
    "ct2d": (["fp64", "fp32"], 0),
    "seismic2d": (["fp64"], 0),
    "dynct": (["fp64", "fp32"], 0),
}


def _steps(eps):
    """eps as a dict of the steps' unit roundoffs (a number applies to every step)."""
    if isinstance(eps, dict):
        return eps
    return {"gradient": eps, "column": eps, "solve": eps, "refine": eps, "combine": eps, "sum": eps}


def _perturbed_aw(P, iters, eps, seed, cgs_passes=2, W0=None):
    """Algorithm 2 with the data flow of the GPU kernels and the roundings of _perturbed: A w of
    every basis column is formed once and kept (A W), the sketched column is S_A applied to that
    stored A w, and every iterate, residual and refinement residual comes from one combine of W
    and A W with the same y (x = W y, e = (A W) y - b; eq. gradient with x = W y).  In exact
    arithmetic this is Algorithm 2; in floating point its rounding differs from the oracle's
    A x - b, so the deviation of these runs from the oracle bounds what two correct
    implementations of the two data flows may differ by.  Built from oracle/ primitives only."""
    import scipy.linalg
    from oracle import sgks_oracle as OS
    rng = np.random.default_rng(seed)
    u = _steps(eps)
    ug, uc, us, ur, ux, um = u["gradient"], u["column"], u["solve"], u["refine"], u["combine"], u["sum"]

    def pert(v, e):
        v = np.asarray(v, dtype=np.float64)
        return v * (1.0 + e * rng.standard_normal(v.shape))

    Aop, Lop = OS.make_operators(P)
    b = np.asarray(P.b, dtype=np.float64)
    lam = float(P.lam)
    SA, SL = OS.sketch_operator(P.sketch, 0, P.m), OS.sketch_operator(P.sketch, 1, P.p)
    Sb = SA @ b
    W = pert(OS.initial_basis(Aop, b, P.ell) if W0 is None else np.array(W0, dtype=np.float64), ug)
    AW = np.zeros((P.m, 0))
    QA, RA = np.zeros((len(Sb), 0)), np.zeros((0, 0))
    QL, RL = np.zeros((SL.shape[0], 0)), np.zeros((0, 0))
    dA = np.zeros(0)

    def append(w):
        nonlocal AW, QA, RA, QL, RL, dA
        aw = Aop.apply(pert(w, um))   # one rounding per term of A w, kept
        AW = np.concatenate([AW, aw[:, None]], axis=1)
        QA, RA, _, _ = OS.qr_append(QA, RA, pert(SA @ aw, uc), cgs_passes)
        QL, RL, _, _ = OS.qr_append(QL, RL, pert(SL @ Lop.apply(w), uc), cgs_passes)
        dA = np.concatenate([dA, [QA[:, -1] @ Sb]])

    def combine(y):   # x = W y and e = (A W) y - b from one rounding per term
        yt = pert(y, ux)
        return W @ yt, AW @ yt - pert(b, um)

    def grad(x, e, u_out):   # eq. gradient from the combined x and e, one rounding per term
        return pert(pert(Aop.adjoint(pert(e, um)), um) + pert(lam * Lop.adjoint(Lop.apply(x)), um), u_out)

    def solve():
        y, T = OS.projected_solve(pert(RA, us), pert(RL, us), pert(dA, us), lam)
        for _ in range(P.n_refine):   # q = 0 refinement: y -= (T^T T)^{-1} W^T r(y)
            x, e = combine(y)
            g = W.T @ grad(x, e, ur)
            t = scipy.linalg.solve_triangular(T, g, trans="T", lower=False)
            y = y - scipy.linalg.solve_triangular(T, t, lower=False)
        return y

    for j in range(W.shape[1]):
        append(W[:, j])
    xs = []
    x, e = combine(solve())
    xs.append(x)
    for _ in range(iters):
        r = grad(x, e, ug)
        W = np.concatenate([W, r[:, None]], axis=1)
        append(r)
        x, e = combine(solve())
        xs.append(x)
    return {"xs": xs}


def floor_curve(P, iters, eps, seeds=5, **kw):
    """(floor_k for k = 0..iters, unperturbed oracle run): the largest relative deviation of
    `seeds` perturbed runs (_perturbed_aw) from the oracle, for problems small enough to run here
    and now.  kw: cgs_passes."""
    import oracle as O
    ref = O.sgks(P, iters=iters, record_x=True, **kw)
    fl = np.zeros(len(ref["xs"]))
    for sd in range(seeds):
        p = _perturbed_aw(P, iters, eps, sd, **kw)
        fl = np.maximum(fl, [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(p["xs"], ref["xs"])])
    return [float(v) for v in fl], ref


def _problem(name, form, params=()):
    """The workload; params may hold sketch_seed, which replaces the sketch seed (a batch shares
    the sketch of its first instance)."""
    from workloads import make_problem
    kw = dict(params)
    sketch_seed = kw.pop("sketch_seed", None)
    P = make_problem(name, **kw)
    if sketch_seed is not None:
        P.sketch.seed = sketch_seed
    if form in ("fp64", "ff"):
        P.n_refine = FORMS[name][1]
    return P


def _parse(target):
    """config[@key=value,...][:form] -> (config, ((key, value), ...), form or None)."""
    head, _, form = target.partition(":")
    name, _, kv = head.partition("@")
    params = tuple((k, int(v)) for k, v in (item.split("=") for item in kv.split(",") if item))
    return name, params, form or None


def _suffix(params):
    return "".join(f"_{k}{v}" for k, v in params)


def _reference(task):
    """The unperturbed oracle run of one target; its iterates go to a scratch file."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    name, params, form, scratch = task
    import oracle as O
    P = _problem(name, form, params)
    ref = O.sgks(P, iters=P.iters, record_x=True)
    np.save(scratch, np.stack([np.asarray(x) for x in ref["xs"]]))
    return [float(v) for v in ref["rre"]]


def _seed(task):
    """One perturbed run of one target against its reference iterates (read from the scratch
    file): the deviation curve."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    name, params, form, scratch, seed = task
    P = _problem(name, form, params)
    p = _perturbed_aw(P, P.iters, EPS[form], seed)
    xs = np.load(scratch, mmap_mode="r")
    return [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(p["xs"], xs)]


def main(argv):
    import tempfile
    ap = argparse.ArgumentParser()
    ap.add_argument("targets", nargs="*")
    ap.add_argument("--seeds", type=int, default=8)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    a = ap.parse_args(argv)
    targets = []
    for t in a.targets or list(FORMS):
        name, params, form = _parse(t)
        for f in ([form] if form else FORMS[name][0]):
            targets.append((name, params, f))
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as tmp, ctx.Pool(a.jobs) as pool:
        scratch = [os.path.join(tmp, f"ref{i}.npy") for i in range(len(targets))]
        rres = pool.map(_reference, [(n, pr, f, sc) for (n, pr, f), sc in zip(targets, scratch)])
        # every (target, seed) pair is one task, so that the seeds of one target run in parallel
        tasks = [(n, pr, f, sc, sd) for (n, pr, f), sc in zip(targets, scratch) for sd in range(a.seeds)]
        curves = pool.map(_seed, tasks)
    for i, ((name, params, form), rre) in enumerate(zip(targets, rres)):
        per_seed = curves[i * a.seeds:(i + 1) * a.seeds]
        floor = [max(c[k] for c in per_seed) for k in range(len(rre))]
        P = _problem(name, form, params)
        out = {"config": name, "params": dict(params), "form": form, "eps": _steps(EPS[form]), "n_refine": P.n_refine,
               "iters": P.iters, "seeds": a.seeds, "floor": floor, "per_seed": per_seed, "oracle_rre": rre,
               "note": "max over seeds of oracle vs oracle with every rounding step perturbed by (1 + u*N(0,1)), "
                       "u per step in eps; written by make_floors.py"}
        with open(os.path.join(HERE, f"floor_{name}{_suffix(params)}_{form}.json"), "w") as f:
            json.dump(out, f)
        print(name + _suffix(params), form, f"floor at k={P.iters}: {floor[-1]:.2e}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
