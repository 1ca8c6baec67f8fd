"""GB300-native HOTRG coarse-graining (Yamashita & Sakurai, arXiv:2110.03607).

The work runs in libhotrg.so (hand-written CUDA for sm_103a, C ABI declared
in include/hotrg.h).  This package is only the ctypes binding, with the same
function names; PyTorch supplies device memory and streams.  There is no CPU
fallback: importing the binding fails if the library is missing.
"""

from .binding import *  # noqa: F401,F403
from .binding import HotrgError, Hotrg, library_path, load  # noqa: F401
