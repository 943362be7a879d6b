"""Plain, slow FP64 CPU oracle for randomized Cholesky QR (Balabanov, arXiv 2210.09953).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library; the two sides meet
only through seeded inputs and the published definitions they both follow.

Modules
-------
philox  Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
theta   The sketching matrix Theta of Sec. 2 realised from Philox bytes.
linalg  Textbook kernels: Householder QR, column-pivoted QR, Cholesky,
        forward substitution, rank test (Alg. 2 step 2, Alg. 3 step 3,
        Alg. 7 steps 2-3).
rcqr    The algorithms: RCholeskyQR (Alg. 2), RCholeskyQR2 (Alg. 3),
        reduced RCholeskyQR (Alg. 5), RRRCholQR (Alg. 7 with the column
        normalisation of Sec. 4) and its CholeskyQR-augmented form, plus
        the stability metrics of Sec. 6.
adjoint Reverse-mode derivative of the RCholeskyQR2 chain (not in the paper).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (published test vectors, closed forms,
textbook/library special cases, invariants of Sec. 5); the one convention
the paper leaves free -- which bit stream realises Theta -- is documented in
``theta`` and is the same definition the library implements independently.
"""
