"""Write tests/golden/floor_<config>_<form>.json: the inherent iterate-agreement floor of sGKS.

sGKS builds its basis from gradients at earlier iterates and never re-orthogonalises, so a
perturbation at the level of rounding grows from one iteration to the next.  Two correct
implementations that differ only in the order of floating-point operations therefore drift
apart.  This script measures that drift with the FP64 oracle alone: it runs the oracle once
unperturbed and then once per seed with every gradient (eq. gradient), every sketched column
entering the QR update (eq. updqr) and the inputs of every projected solve multiplied entrywise
by (1 + eps * N(0,1)) -- the backward errors of those steps -- and records, for every k, the
largest ||x_k - x'_k|| / ||x'_k|| over the seeds (five by default).  eps = 2^-53 models FP64 arithmetic, eps = 2^-48 float-float
arithmetic (a 48-bit significand), eps = 2^-24 FP32 storage of the basis.  The per-seed curves are kept too.  The parity tests accept a CUDA iterate when its error
against the oracle is below max(tolerance, FACTOR * floor_k).

Only oracle/ and workloads/ are used.  Run:
    python tests/golden/make_floors.py [config[@key=value,...][:form] ...] [--seeds N] [--jobs J]
A target such as ct2d@instance=21:ff passes instance=21 to the workload generator and writes
floor_ct2d_instance21_ff.json (the batched tests compare single instances of a batch).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

EPS = {"fp64": 2.0 ** -53, "ff": 2.0 ** -48, "fp32": 2.0 ** -24}
FORMS = {  # config -> (forms, n_refine used with the FP64 and float-float forms)
    "deconv1d": (["fp64"], 0),
    "deblur2d": (["fp64", "fp32"], 0),
    "ct2d": (["fp64", "fp32"], 0),
    "seismic2d": (["fp64"], 0),
    "dynct": (["fp64", "fp32"], 0),
}


def _perturbed(P, iters, eps, seed, **kw):
    """Oracle iterates of a nearby computation: every gradient (eq. gradient), every sketched
    column entering the QR update (eq. updqr) and the inputs R_A, R_L, d_A of each projected
    solve (eq. projected_sketched_bis) multiplied entrywise by (1 + eps N(0,1)), seeded.  Each of
    these steps is backward stable, so a correct implementation computes the exact result of
    such a nearby input; the perturbation models the rounding of every one of them."""
    import oracle as O
    from oracle import sgks_oracle as OS
    rng = np.random.default_rng(seed)
    orig_g, orig_qr, orig_ps = OS.gradient, OS.qr_append, OS.projected_solve

    def pert(v):
        v = np.asarray(v, dtype=np.float64)
        return v * (1.0 + eps * rng.standard_normal(v.shape))

    OS.gradient = lambda A, L, b, lam, x: pert(orig_g(A, L, b, lam, x))
    OS.qr_append = lambda Q, R, u, passes=2, breakdown_tol=1e-13: orig_qr(Q, R, pert(u), passes, breakdown_tol)
    OS.projected_solve = lambda RA, RL, dA, lam: orig_ps(pert(RA), pert(RL), pert(dA), lam)
    try:
        return O.sgks(P, iters=iters, record_x=True, **kw)
    finally:
        OS.gradient, OS.qr_append, OS.projected_solve = orig_g, orig_qr, orig_ps


def floor_curve(P, iters, eps, seeds=5, **kw):
    """(floor_k for k = 0..iters, unperturbed oracle run): the largest relative deviation over
    `seeds` perturbed runs, for problems small enough to run here and now.  kw: options of
    oracle.sgks (e.g. cgs_passes)."""
    import oracle as O
    ref = O.sgks(P, iters=iters, record_x=True, **kw)
    fl = np.zeros(len(ref["xs"]))
    for sd in range(seeds):
        p = _perturbed(P, iters, eps, sd, **kw)
        fl = np.maximum(fl, [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(p["xs"], ref["xs"])])
    return [float(v) for v in fl], ref


def _problem(name, form, params=()):
    from workloads import make_problem
    P = make_problem(name, **dict(params))
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


def _run(task):
    """One target (config, parameters, form) in one process: the unperturbed oracle run, then one
    perturbed run per seed, keeping only the deviation curves (the iterates of one run at a time)."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    name, params, form, seeds = task
    import oracle as O
    P = _problem(name, form, params)
    ref = O.sgks(P, iters=P.iters, record_x=True)
    xs = [np.asarray(x) for x in ref["xs"]]
    rre = [float(v) for v in ref["rre"]]
    del ref
    curves = []
    for sd in range(seeds):
        p = _perturbed(P, P.iters, EPS[form], sd)
        curves.append([float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(p["xs"], xs)])
        del p
    return task, curves, rre


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("targets", nargs="*")
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    a = ap.parse_args(argv)
    targets = []
    for t in a.targets or list(FORMS):
        name, params, form = _parse(t)
        for f in ([form] if form else FORMS[name][0]):
            targets.append((name, params, f))
    tasks = [(n, pr, f, a.seeds) for n, pr, f in targets]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(a.jobs, len(tasks))) as pool:
        for (name, params, form, seeds), curves, rre in pool.imap_unordered(_run, tasks):
            floor = [max(c[k] for c in curves) for k in range(len(rre))]
            P = _problem(name, form, params)
            out = {"config": name, "params": dict(params), "form": form, "eps": EPS[form], "n_refine": P.n_refine,
                   "iters": P.iters, "seeds": seeds, "floor": floor, "per_seed": curves, "oracle_rre": rre,
                   "note": "max over seeds of oracle vs oracle with gradients, sketched QR inputs and projected-solve "
                           "inputs perturbed by (1 + eps*N(0,1)); written by make_floors.py"}
            with open(os.path.join(HERE, f"floor_{name}{_suffix(params)}_{form}.json"), "w") as f:
                json.dump(out, f)
            print(name + _suffix(params), form, f"floor at k={P.iters}: {floor[-1]:.2e}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
