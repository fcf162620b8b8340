"""GB300-native hot path of the BBMD short-range molecular-dynamics method: a C-ABI CUDA
library (csrc/, include/bbmd.h) and its thin ctypes binding (bbmd.py)."""
from . import bbmd  # noqa: F401
