"""Plain FP64 CPU oracle for the one-obstacle MFS solution operator.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package. The product path
(`paper_1506_05083_gb300`) never imports, calls or links it, and this package
never imports the product: the two share only the seeded workload
descriptions in `synth/`.

Every function follows the paper's statement of the method directly: direct
summation in place of FFTs, unblocked Householder QR, plain back substitution,
no blocking or reordering. Each function cites the section or equation it
restates. Parity status of each function (what pins it) is listed in
`oracle/mfs.py`'s module docstring; the periodizing scheme's spherical-wave
block B~ (Sec. 4.1) is in `oracle/periodizing.py`, with its own pins.
"""
from .mfs import *  # noqa: F401,F403
from . import periodizing  # noqa: F401
