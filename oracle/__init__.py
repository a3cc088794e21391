"""FP64 CPU oracle for the augmented FEWHA hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the GPU library computes (Ramlau & Stadler, Sec. 2-4,
Algorithms 1-3).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
library and never imports it; the library never imports this package.

Parity status of each function (what pins it) is listed in the module
docstrings and in the test files ``tests/test_oracle_*.py``.
"""
from .oracle import Oracle, build_oracle, oracle_lib_path  # noqa: F401
from .daubechies import daubechies_taps  # noqa: F401
