"""FP64 CPU oracle for the randomized QB / RSVD / ID / CUR path.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library package never
does, and it shares no code, tables or helpers with the CUDA sources.

Contents
--------
philox   counter-based Philox4x32-10 stream and the Box-Muller Gaussian test
         matrix Omega (written from Salmon et al., SC'11, and Box & Muller 1958).
rsvd     the algorithms of Voronin & Martinsson (RSVDPACK), step by step in
         FP64: orth (Householder QR), the range finder with power scheme,
         the QB step, Algorithm 5 (RSVD version II), k-step column-pivoted QR,
         the QB-route randomized ID, the CUR of Algorithm 3, the blocked
         adaptive QB to a tolerance of Algorithm 7, the parallel blocked QB of
         Algorithm 8, the randomized ID from the left sketch (Sec. 3.5) and
         the reverse-mode derivative of Algorithm 5 with Omega fixed.
jacobi   the one-sided Jacobi SVD (Hestenes) of the l x l core of Alg. 5,
         round-robin pair order, Demmel-Veselic stopping rule.
quant    the E4M3 format, its round-to-nearest-even quantiser with block
         scales, and the FP8 sketch of the dequantised operands (the reading
         of the FP8 sketch; the paper fixes no reduced precision).
"""
from . import jacobi, philox, quant, rsvd  # noqa: F401
