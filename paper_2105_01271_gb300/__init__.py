"""GB300 (sm_103a) deterministic-sketch low-rank compression.

The compute lives in the CUDA library liblrs.so (C ABI: include/lrs.h),
built by ``build.build()``; ``binding`` is its thin ctypes wrapper and
``path`` composes the C-ABI calls of the paper's hot path.  Importing this
package does not load the library; ``binding.load()`` does, and fails loudly
if it cannot.
"""
__all__ = ["binding", "build", "path"]
