"""GB300 (sm_103a) implementation of the chaotic video cipher of arXiv 2302.07411.

The compute lives in ``libvcrypt.so`` (CUDA kernels behind the C ABI of
``include/vcrypt.h``); ``binding`` is its thin ctypes binding.  Importing this
package does not load the library; ``binding.lib()`` does, and raises when the
library has not been built.
"""
__all__ = ["binding", "build"]
