"""GB300 library for the implicit theta-weighted step on the adaptive polar mesh of
the unit disk (parabolic and drift-diffusion equations).  The compute path is the CUDA
library libpolar.so (C ABI in include/polar.h); this package only marshals arguments."""
from ._native import *  # noqa: F401,F403
from ._native import load, LIB_PATH, EXPORTS, PolarError, Ctx  # noqa: F401
