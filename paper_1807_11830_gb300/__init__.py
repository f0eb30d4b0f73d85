"""GB300-native multi-coil Cartesian SENSE (arXiv 1807.11830, Eq. 1 and the
CG-SENSE reconstruction built on it).

The compute path lives in the CUDA library ``libsense.so`` behind the C ABI
declared in ``include/sense.h``; ``paper_1807_11830_gb300.sense`` is its thin
Python binding.  Importing this package loads nothing; the first call into
the binding loads the library and raises if it has not been built.
"""
__all__ = ["sense", "synth"]
