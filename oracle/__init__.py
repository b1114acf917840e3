"""FP64 CPU oracle for blockBP (arXiv:2301.05844).

Test infrastructure only: used by tests/, __graft_entry__.smoke() and the CPU
baseline legs of bench.py.  The CUDA library never imports or runs it.
"""
