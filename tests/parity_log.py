"""Records of the iterate comparisons made by the GPU parity tests.

Each check stores, for one run, the largest error against the oracle, the largest ratio of that
error to the method's own floor, and the last iteration at which the strict bar still held.  When
SGKS_PARITY_LOG names a file, tests/conftest.py writes the records there as JSON at the end of the
session (these are the figures behind the tolerance factors)."""
import numpy as np

RECORDS = []


def record(name, errs, floor, tol, factor):
    errs = [float(e) for e in errs]
    fl = [float(f) for f in floor[:len(errs)]]
    ratios = [e / f for e, f in zip(errs, fl) if f > 0 and e > tol]
    k_strict = max([k for k, e in enumerate(errs) if e < tol] + [0])
    RECORDS.append({"name": name, "iters": len(errs) - 1, "max_err": max(errs), "final_err": errs[-1],
                    "max_ratio_to_floor_above_tol": max(ratios) if ratios else 0.0, "tol": tol,
                    "factor": factor, "strict_through": k_strict,
                    "floor_final": fl[-1] if len(fl) == len(errs) else None,
                    "errs": errs if len(errs) > 40 else None, "floor": fl if len(errs) > 40 else None})
    return errs


def max_ratio():
    return max([r["max_ratio_to_floor_above_tol"] for r in RECORDS] + [0.0])


def summary():
    return {"records": RECORDS, "max_ratio": max_ratio(),
            "count": len(RECORDS), "median_ratio": float(np.median([r["max_ratio_to_floor_above_tol"]
                                                                     for r in RECORDS])) if RECORDS else 0.0}
