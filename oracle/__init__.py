"""CPU oracle for Zolo-PD / Zolo-SVD: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The CUDA library and its binding never call it.
"""
