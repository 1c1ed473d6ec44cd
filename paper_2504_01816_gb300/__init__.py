"""GB300 (sm_103a) implementation of the hot path of the real-space RPA correlation-energy
method (arXiv 2504.01816): batched Sternheimer COCG, Kronecker-product Coulomb operator,
subspace iteration with Rayleigh-Ritz.  The computation lives in librpa.so (include/rpa.h);
this package is its ctypes binding."""
from .rpa import *  # noqa: F401,F403
from .rpa import Context, Options, EcResult, RpaError, default_options, library, LIB_PATH, EXPORTED  # noqa: F401
