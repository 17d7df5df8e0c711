"""GB300 (sm_103a) one-obstacle MFS solution operator (arXiv:1506.05083).

The compute path is the CUDA library libaxi_mfs.so (C ABI in
include/axi_mfs.h); `axi` is its thin ctypes binding.
"""
from . import axi  # noqa: F401
from .axi import Operator, ObstacleSpec, geometry, choose_q, spec_from_obstacle  # noqa: F401
