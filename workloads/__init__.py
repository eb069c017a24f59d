"""Seeded synthetic inputs for the sGKS workloads.

This package holds the input generators that both the FP64 oracle (``oracle/``)
and the CUDA library are fed from.  It contains none of the method's arithmetic:
it only builds problem data (operators A and L as descriptors, x_true, b,
lambda, sketch sizes, Gaussian sketch matrices where a config asks for them).

The workloads are stand-ins shaped like the paper's experiments (Sec. 4: image
deblurring, X-ray CT, seismic travel-time tomography, dynamic CT); the paper's
own datasets are not available, so every array is generated from a seed.
"""
from .problem import Problem, OperatorDesc, RegDesc, SketchDesc
from .configs import CONFIG_NAMES, make_problem, small_problem

__all__ = [
    "Problem", "OperatorDesc", "RegDesc", "SketchDesc",
    "CONFIG_NAMES", "make_problem", "small_problem",
]
