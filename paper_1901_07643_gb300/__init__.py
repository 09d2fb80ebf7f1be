"""GB300 library for the all-families regression scores of arXiv 1901.07643.

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python names here only marshal arguments to its C entry points.  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
