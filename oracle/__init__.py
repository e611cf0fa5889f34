"""CPU reference (oracle) for the batched tridiagonal solve. TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package. The CUDA library never calls it and shares no code with it.
"""
from .tdma_oracle import *  # noqa: F401,F403
