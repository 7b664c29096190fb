"""GB300-native multilevel entropic-risk gradient engine (libmlsgd + binding).

The compute path lives in the CUDA library ``libmlsgd.so`` built from
``csrc/`` (see ``include/mlsgd.h``); ``mlsgd`` is its ctypes binding.
"""
from . import inputs  # noqa: F401
