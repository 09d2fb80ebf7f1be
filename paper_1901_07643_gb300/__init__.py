"""GB300 library for the all-families regression scores of arXiv 1901.07643.

The compute path lives in the CUDA shared library built from ``csrc/``
(``python -m paper_1901_07643_gb300.build``); the names exported here only
marshal arguments to its C entry points (``include/givensbn.h``).  Importing
the package does not load the library; the first call does, and raises if it
has not been built.
"""
from .binding import (GivensBNError, all_family_scores, auto_q, autotune,  # noqa: F401
                      autotune_batched, batch_offsets, backward_workspace_size, best_parents,
                      batched_workspace_size, family_coefficients, load, plan_choice,
                      score_all_families, score_all_families_batched,
                      score_all_families_backward, score_all_families_backward_batched,
                      score_all_families_noalloc, shard_range,
                      strerror, structure_search, workspace_size)
