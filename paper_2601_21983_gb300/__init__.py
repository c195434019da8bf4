"""GB300 (sm_103a) implementation of the data-annealed SMC sampler for
neural-network posteriors.  The compute lives in libsmc.so (CUDA kernels behind
the C ABI of include/smc.h); `smc` is its Python binding."""
from . import smc  # noqa: F401

__all__ = ["smc"]
