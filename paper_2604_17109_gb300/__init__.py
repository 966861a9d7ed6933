"""GB300-native PIMI sweep library (probabilistic Ising machine with inertia).

The compute lives in ``libpimi.so`` (CUDA for sm_103a); ``pim`` is its ctypes binding.
"""
from . import pim  # noqa: F401
