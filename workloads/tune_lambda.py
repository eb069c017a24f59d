"""Grid search of the regularisation parameter with the FP64 oracle (the paper hand-tunes
lambda* to minimise the final RRE, Sec. 4).  Used for the configs that state no lambda
(seismic2d, dynct); the chosen values are frozen in workloads/configs.py.

Run:  python workloads/tune_lambda.py seismic2d 1e-1 1e3   (15 log-spaced values, 8 processes)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _rre(args):
    name, lam = args
    import oracle as O
    from workloads import make_problem
    P = make_problem(name, lam=lam)
    return lam, float(O.sgks(P)["rre"][-1])


def main(name, lo, hi, count=15, procs=8):
    grid = np.logspace(np.log10(lo), np.log10(hi), count)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = sorted(pool.map(_rre, [(name, float(l)) for l in grid]))
    for lam, r in res:
        print(f"{name} lambda={lam:.4g} final RRE={r:.5f}")
    best = min(res, key=lambda t: t[1])
    print(f"{name} best lambda={best[0]:.4g} RRE={best[1]:.5f}")


if __name__ == "__main__":
    main(sys.argv[1], float(sys.argv[2]), float(sys.argv[3]))
