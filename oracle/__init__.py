"""Plain, slow FP64 CPU oracle of the rank-structured supernodal Cholesky
preconditioner (Chadwick & Bindel, "An efficient solver for sparse linear
systems based on rank-structured Cholesky factorization", arXiv 1507.05593).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports or calls this
package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do.  It shares no code with the CUDA path (``paper_1507_05593_gb300``):
the only module both sides read is the input generator ``workloads``.

Each function follows one passage of the paper, in the paper's order and
notation, with numpy arrays; dense Cholesky, triangular solves and the
Householder QR are written out as loops (``oracle.dense``).  Where the paper is
silent, garbled or inconsistent, the reading taken is stated at the function.

Pins (tests/test_oracle_*.py) tie every part to something other than itself:
the worked scatter example of Section 2.1, brute-force symbolic elimination,
dense Cholesky of the permuted matrix, explicitly formed blocks, dense SVDs,
the Philox known-answer vectors and PCG residuals.

Parity status per function is stated in its docstring; every function listed
in ``__all__`` of the submodules is pinned.
"""
