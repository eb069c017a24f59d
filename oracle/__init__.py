"""FP64 CPU oracle for sGKS -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg may import it; the library itself never does, and the
oracle imports nothing from the library.  It shares no code with the CUDA path.

Parity status per function is stated in each module's header.
"""
from .sgks_oracle import (  # noqa: F401
    splitmix64_mix,
    sparse_sign_rows,
    sketch_operator,
    make_operators,
    initial_basis,
    qr_append,
    projected_solve,
    refine_step,
    sgks,
    gks,
    tikhonov_functional,
    direct_solve,
)
