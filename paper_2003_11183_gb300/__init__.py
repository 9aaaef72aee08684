"""GB300 (sm_103a) tile-low-rank quasi-Monte Carlo library for high-dimensional
multivariate normal and Student-t probabilities.  The CUDA library is
libtlrmvn.so (C ABI in include/tlrmvn.h); ``api`` is its Python binding."""
from .api import *  # noqa: F401,F403
from .api import Factor, TlrmvnError, ExportedFactor, parse_export, build_export  # noqa: F401
