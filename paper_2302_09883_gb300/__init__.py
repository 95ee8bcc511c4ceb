"""wcsim: wavelet-compressed patch time stepping of LBM/FV schemes on GB300.

Import is cheap; the CUDA library is loaded (and must exist) when a Sim or
Dense is created.
"""
from .sim import Dense, Dense3, Sim, Sim3  # noqa: F401
from .batch import Batch, autotune  # noqa: F401
from . import inputs  # noqa: F401
