"""CPU oracle for recursive fast matrix multiplication (Benson & Ballard,
"A Framework for Practical Parallel Fast Matrix Multiplication").

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__
and the CPU-baseline leg of bench.py may import or run anything here.  It
shares no code with the GPU library and imports nothing from it.

Contents
  classical.c / _native.py  classical FP64 product C = A B (Section 2.1),
                            plus long-double and per-entry variants
  tensor.py                 matmul tensor (Section 2.2.2), exact Brent check
                            (Eq. 2), L-level flattening, Props 2.1 and 2.2
  fastmm.py                 recursive fast multiply, write-once additions,
                            top-level peeling (Sections 3.1, 3.2, 3.5)
  norms.py                  error norms e_F and e_max
  costs.py                  flop, addition and traffic models (Sections 2.1,
                            3.2, 4.2, Table 1)
"""
from . import _native, costs, fastmm, norms, tensor  # noqa: F401
from ._native import gemm, gemm_entries  # noqa: F401
