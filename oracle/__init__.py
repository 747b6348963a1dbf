"""FP64 CPU oracle of the FDLB time step (arXiv:1010.4124).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It shares
no code with the CUDA path (paper_1010_4124_gb300) and never imports it.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, textbook special cases or brute force; none is
"parity unpinned".
"""
