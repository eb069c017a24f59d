"""Write tests/golden/floor_<config>_<form>.json: the inherent iterate-agreement floor of sGKS.

sGKS builds its basis from gradients at earlier iterates and never re-orthogonalises, so a
perturbation at the level of rounding grows from one iteration to the next.  Two correct
implementations that differ only in the order of floating-point operations therefore drift
apart.  This script measures that drift with the FP64 oracle alone: it runs the oracle once
unperturbed and then once per seed with every gradient (eq. gradient) multiplied entrywise by
(1 + eps * N(0,1)), and records, for every k, the largest ||x_k - x'_k|| / ||x'_k|| over the
seeds (five by default).  eps = 2^-53 models FP64 arithmetic, eps = 2^-48 float-float
arithmetic (a 48-bit significand), eps = 2^-24 FP32 storage of the basis.  The per-seed curves are kept too.  The parity tests accept a CUDA iterate when its error
against the oracle is below max(tolerance, FACTOR * floor_k).

Only oracle/ and workloads/ are used.  Run:
    python tests/golden/make_floors.py [config[:form] ...] [--seeds N] [--jobs J]
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
FORMS = {  # config -> (forms, n_refine used with the FP64 form)
    "deconv1d": (["fp64"], 0),
    "deblur2d": (["fp64", "fp32"], 0),
    "ct2d": (["fp64", "fp32"], 0),
    "seismic2d": (["fp64"], 0),
    "dynct": (["fp64", "fp32"], 0),
}


def _perturbed(P, iters, eps, seed):
    """Oracle iterates with every gradient multiplied entrywise by (1 + eps N(0,1)) (seeded)."""
    import oracle as O
    from oracle import sgks_oracle as OS
    rng = np.random.default_rng(seed)
    orig = OS.gradient

    def pert(A, L, b, lam, x):
        r = orig(A, L, b, lam, x)
        return r * (1.0 + eps * rng.standard_normal(r.shape))

    OS.gradient = pert
    try:
        return O.sgks(P, iters=iters, record_x=True)
    finally:
        OS.gradient = orig


def floor_curve(P, iters, eps, seeds=5):
    """(floor_k for k = 0..iters, unperturbed oracle run): the largest relative deviation over
    `seeds` perturbed runs, for problems small enough to run here and now."""
    import oracle as O
    ref = O.sgks(P, iters=iters, record_x=True)
    fl = np.zeros(len(ref["xs"]))
    for sd in range(seeds):
        p = _perturbed(P, iters, eps, sd)
        fl = np.maximum(fl, [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(p["xs"], ref["xs"])])
    return [float(v) for v in fl], ref


def _problem(name, form):
    from workloads import make_problem
    P = make_problem(name)
    if form == "fp64":
        P.n_refine = FORMS[name][1]
    return P


def _run(task):
    """One oracle run of (config, form) with the gradients perturbed by `seed` (None: unperturbed)."""
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    name, form, seed = task
    import oracle as O
    P = _problem(name, form)
    if seed is None:
        ref = O.sgks(P, iters=P.iters, record_x=True)
        return task, [np.asarray(x) for x in ref["xs"]], [float(v) for v in ref["rre"]]
    p = _perturbed(P, P.iters, EPS[form], seed)
    return task, [np.asarray(x) for x in p["xs"]], None


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("targets", nargs="*")
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    a = ap.parse_args(argv)
    targets = []
    for t in a.targets or list(FORMS):
        name, _, form = t.partition(":")
        for f in ([form] if form else FORMS[name][0]):
            targets.append((name, f))
    tasks = [(n, f, s) for n, f in targets for s in [None] + list(range(a.seeds))]
    ctx = mp.get_context("spawn")
    results = {}
    with ctx.Pool(a.jobs) as pool:
        for task, xs, rre in pool.imap_unordered(_run, tasks):
            results[task] = (xs, rre)
    for name, form in targets:
        ref, rre = results[(name, form, None)]
        curves = []
        for s in range(a.seeds):
            xs = results[(name, form, s)][0]
            curves.append([float(np.linalg.norm(x - r) / np.linalg.norm(r)) for x, r in zip(xs, ref)])
        floor = [max(c[k] for c in curves) for k in range(len(ref))]
        P = _problem(name, form)
        out = {"config": name, "form": form, "eps": EPS[form], "n_refine": P.n_refine, "iters": P.iters,
               "seeds": a.seeds, "floor": floor, "per_seed": curves, "oracle_rre": rre,
               "note": "max over seeds of oracle vs oracle with gradients perturbed by (1 + eps*N(0,1)); "
                       "written by make_floors.py"}
        with open(os.path.join(HERE, f"floor_{name}_{form}.json"), "w") as f:
            json.dump(out, f)
        print(name, form, f"floor at k={P.iters}: {floor[-1]:.2e}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
