"""GB300-native sGKS: the per-iteration hot path of the sketched generalized Krylov subspace
method for Tikhonov regularization, as hand-written CUDA kernels for sm_103a behind a C ABI
(include/sgks.h), with this thin Python binding on top.

    from paper_2606_18073_gb300 import Solver, CSR, Dense, Conv2D, Reg
"""
from . import _lib
from .solver import (PRECISIONS, Batch, CSR, Conv2D, Dense, Reg, SGKSFunction, Solver, device_inputs, io_dtype,
                     kernel_launches, solve_differentiable, sparse_sign_rows)

__all__ = ["Solver", "Batch", "SGKSFunction", "solve_differentiable", "CSR", "Dense", "Conv2D", "Reg", "device_inputs", "kernel_launches", "sparse_sign_rows", "io_dtype", "PRECISIONS", "_lib", "build"]


def build(force: bool = False) -> str:
    """Compile libsgks.so in-tree for sm_103a and load it."""
    from ._build import build as _b
    path = _b(force=force)
    _lib.load(path)
    return path
