"""Write tests/golden/floor_<config>_<form>.json: the inherent iterate-agreement floor of sGKS.

sGKS builds its basis from gradients at earlier iterates and never re-orthogonalises, so a
perturbation at the level of rounding grows from one iteration to the next.  Two correct
implementations that differ only in the order of floating-point operations therefore drift
apart.  This script measures that drift with the FP64 oracle alone: it runs the oracle twice
on the same problem, the second time with every gradient (eq. gradient) multiplied entrywise
by (1 + eps * N(0,1)), and records ||x_k - x'_k|| / ||x'_k|| for every k.  eps = 2^-53 models
FP64 arithmetic, eps = 2^-24 FP32 arithmetic.  The parity tests accept a CUDA iterate when its
error against the oracle is below max(tolerance, FACTOR * floor_k).

Only oracle/ and workloads/ are used.  Run:  python tests/golden/make_floors.py [config ...]
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from oracle import sgks_oracle as OS  # noqa: E402
from workloads import make_problem  # noqa: E402

EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
FORMS = {  # config -> (forms, n_refine used with the FP64 form)
    "deconv1d": (["fp64"], 0),
    "deblur2d": (["fp64", "fp32"], 0),
    "ct2d": (["fp64"], 0),
    "seismic2d": (["fp64"], 0),
    "dynct": (["fp64", "fp32"], 0),
}


def floor_curve(P, iters, eps, seed=0):
    ref = O.sgks(P, iters=iters, record_x=True)
    rng = np.random.default_rng(seed)
    orig = OS.gradient

    def pert(A, L, b, lam, x):
        r = orig(A, L, b, lam, x)
        return r * (1.0 + eps * rng.standard_normal(r.shape))

    OS.gradient = pert
    try:
        p = O.sgks(P, iters=iters, record_x=True)
    finally:
        OS.gradient = orig
    return [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(p["xs"], ref["xs"])], ref


def main(names):
    for name in names:
        forms, nref64 = FORMS[name]
        for form in forms:
            P = make_problem(name)
            if form == "fp64":
                P.n_refine = nref64
            curve, ref = floor_curve(P, P.iters, EPS[form])
            out = {"config": name, "form": form, "eps": EPS[form], "n_refine": P.n_refine, "iters": P.iters,
                   "floor": curve, "oracle_rre": [float(v) for v in ref["rre"]],
                   "note": "oracle vs oracle with gradients perturbed by (1 + eps*N(0,1)); written by make_floors.py"}
            path = os.path.join(HERE, f"floor_{name}_{form}.json")
            with open(path, "w") as f:
                json.dump(out, f)
            print(name, form, f"floor at k={P.iters}: {curve[-1]:.2e}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(FORMS))
