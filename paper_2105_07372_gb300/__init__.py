"""GB300 (sm_103a) Synch-EM for 2-D multi-reference alignment.

The computation lives in libmra.so (CUDA, C ABI in include/mra.h); ``mra`` is
its ctypes binding, ``pipeline`` strings the calls into the Synch-EM
algorithm, ``autograd`` wraps the marginal log-likelihood and its gradient.
"""
from . import mra  # noqa: F401
