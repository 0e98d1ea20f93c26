"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module builds input matrices only; it holds none of the randomized
algorithm's arithmetic (no sketch, no orthonormalisation of samples, no SVD of
B).  The random Gaussian test matrix Omega is NOT made here: each side draws it
from the Philox counter stream on its own.

Test matrices follow the recipe of Sec. 5 of the paper: A = U D V^* with U and
V random matrices with orthonormal columns (orthonormalised i.i.d. N(0,1)
matrices) and D a prescribed decaying spectrum, plus optional i.i.d. Gaussian
noise of standard deviation ``noise``.
"""
from .matrices import (CONFIGS, config, spectrum, make_matrix_np,  # noqa: F401
                       make_matrix_torch, low_rank_np, BATCH_CONFIGS, batch_sizes,
                       make_batch_torch)
