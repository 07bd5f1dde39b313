"""csfast: GB300-native fast correlation for matching pursuit (arXiv 1205.4139).

The compute path is the CUDA library ``libcsfast.so`` (sources in ``csrc/``,
C ABI declared in ``include/csfast.h``).  ``binding`` wraps that C ABI with
ctypes; it loads the library lazily and raises if it is missing.  There is no
CPU fallback.
"""
__all__ = ["binding", "costmodel"]
