"""CPU oracle (plain FP64 numpy) for the reactive two-phase LBM step.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark.  The product library never imports, links or
calls anything in this package.

Pinned functions and their pins are listed in the design notes; the coupled
multiphase run as a whole has no closed form ("parity unpinned" beyond its
invariants), so it is pinned through its parts.
"""
from .lbm import *  # noqa: F401,F403
from .lbm import Lattice, splitmix64, overflow_key  # noqa: F401
