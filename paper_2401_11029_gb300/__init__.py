"""GB300-native CFL-reachability solver (matrix-based algorithm, arXiv 2401.11029).

The product is the C-ABI library ``libcflr.so`` (include/cflr.h): a WCNF
grammar compiler in C++ and the semi-naive closure loop of the paper's
Algorithm 1 as CUDA kernels for sm_103a.  ``cflr`` is its Python binding
(same function names); ``gen`` makes the seeded synthetic inputs.
"""
from .cflr import (CFLR_FORM_BATCHED, CFLR_FORM_GRAPH, CFLR_FORM_PLAIN, CflrError, Solver,  # noqa: F401
                   cflr_create, cflr_default_config, cflr_destroy, cflr_get_pairs,
                   cflr_autotune, cflr_get_pairs_device, cflr_get_tuning, cflr_set_tuning, cflr_grammar_sizes, cflr_kernel_stats, cflr_reset, cflr_last_error, cflr_load_grammar,
                   cflr_load_graph, cflr_solve, cflr_solve_batch, cflr_symbol_id, load_library)
