"""FP64 CPU oracle of the Fast Finite Shearlet Transform (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA product path never does.
"""
from . import ffst_oracle  # noqa: F401
