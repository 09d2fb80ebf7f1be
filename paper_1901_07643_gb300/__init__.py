"""GB300 library for the all-families regression scores of arXiv 1901.07643.

The compute path lives in the CUDA shared library built from ``csrc/``
(``python -m paper_1901_07643_gb300.build``); the names exported here only
marshal arguments to its C entry points (``include/givensbn.h``).  Importing
the package does not load the library; the first call does, and raises if it
has not been built.
"""
from .binding import (GivensBNError, auto_q, load, score_all_families,  # noqa: F401
                      score_all_families_noalloc, strerror, workspace_size)
