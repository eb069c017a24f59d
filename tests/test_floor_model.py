"""Pins of the sensitivity-floor model (tests/golden/make_floors.py), CPU only.

The floors that gate the GPU parity tests come from Algorithm 2 run in the data flow of the GPU
kernels (A w kept per basis column, e = (A W) y - b) with rounding-level perturbations, against the
oracle's iterates.  These tests check that model against what it must satisfy: with no
perturbation it is Algorithm 2 (it agrees with oracle.sgks to rounding, so a dropped term, a wrong
sign or a transposed operand in it would show), its deviation grows with the unit roundoff, and
a perturbation of the same size in every step gives seeded, reproducible curves."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from workloads import small_problem

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_floors import EPS, _perturbed_aw, floor_curve  # noqa: E402


def rel_dev(xs, ref):
    return [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(xs, ref)]


@pytest.mark.parametrize("kind", ["ct2d", "deblur2d", "seismic2d", "deconv1d", "dynct"])
def test_unperturbed_data_flow_is_algorithm_2(kind):
    """u = 0: the kernels' data flow (e = (A W) y - b, sketched columns from the kept A w, the
    q = 0 refinement from the same combine) reproduces the oracle's iterates up to rounding."""
    P = small_problem(kind)
    ref = O.sgks(P, record_x=True)["xs"]
    xs = _perturbed_aw(P, P.iters, 0.0, 0)["xs"]
    assert len(xs) == len(ref) == P.iters + 1
    assert max(rel_dev(xs, ref)) < 1e-9


def test_planted_mistake_in_the_data_flow_is_visible():
    """A wrong regularization parameter inside the data-flow run (lambda doubled) moves the
    iterates far beyond any floor: the zero-perturbation check above would catch such a slip."""
    P = small_problem("ct2d")
    ref = O.sgks(P, record_x=True)["xs"]
    Q = small_problem("ct2d")
    Q.lam = 2.0 * P.lam
    xs = _perturbed_aw(Q, Q.iters, 0.0, 0)["xs"]
    assert max(rel_dev(xs, ref)) > 1e-4


def test_floor_grows_with_the_unit_roundoff_and_is_seeded():
    P = small_problem("seismic2d")
    f53, _ = floor_curve(P, P.iters, EPS["fp64"], seeds=2)
    f48, _ = floor_curve(P, P.iters, {k: 2.0 ** -48 for k in EPS["fp64"]}, seeds=2)
    again, _ = floor_curve(P, P.iters, EPS["fp64"], seeds=2)
    assert f53 == again                  # seeded: the same curve twice
    assert f48[-1] > 4.0 * f53[-1]       # 32x the roundoff: a clearly larger floor
    assert all(v >= 0.0 for v in f53)
