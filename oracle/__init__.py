"""FP64 CPU oracle for the finite element weak-form evaluator (test infrastructure).

Only the tests, the package smoke check and the CPU-baseline leg of the
benchmark may import this package.  See oracle.c for the definitions.
"""
from .oracle import *  # noqa: F401,F403
