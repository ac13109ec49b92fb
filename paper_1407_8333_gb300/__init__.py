"""GB300-native frequency-Hough transform (Astone et al., arXiv:1407.8333).

The compute path is the C-ABI library ``libfh`` (hand-written sm_103a CUDA,
declared in ``include/fh.h``); ``paper_1407_8333_gb300.fh`` is its thin ctypes
binding with the same entry-point names.  ``synth`` holds the seeded synthetic
input generators.  Importing the package loads nothing; the library is loaded
on first use of the binding and fails loudly when it is missing.
"""
__all__ = ["fh", "synth", "build"]
