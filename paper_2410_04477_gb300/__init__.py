"""GB300-native block-Vecchia Gaussian-process log-likelihood (arXiv 2410.04477).

The compute path is the CUDA library ``libbv.so`` (C ABI declared in ``include/bv.h``);
``paper_2410_04477_gb300.bv`` is its thin ctypes binding.  Importing this package does
not load the library; ``bv`` raises if the library is missing or was not built.
"""
__all__ = ["bv", "synth"]
