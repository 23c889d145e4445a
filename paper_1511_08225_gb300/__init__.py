"""GB300 speed-limited particle-in-cell (SLPIC, arXiv 1511.08225), 1D3V electrostatic.

The simulation runs in the CUDA library ``libslpic.so`` (C ABI in
``include/slpic.h``); this package holds its build script, a thin ctypes
binding with the same entry-point names, and seeded synthetic inputs.
"""
from . import inputs  # noqa: F401
from .binding import *  # noqa: F401,F403
from .binding import EXPORTS, LIB_PATH, Simulation, SlpicError, load_library  # noqa: F401
