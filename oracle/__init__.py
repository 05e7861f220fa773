"""FP64 CPU oracle of the Greedy Frank-Wolfe method -- test infrastructure only.

Imported by the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py`; never by the CUDA library or its Python binding.
"""
from .gfw import *  # noqa: F401,F403
