"""Plain, slow FP64 CPU oracle of the FFT-accelerated surface BIE method.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke()
and by the CPU-baseline leg of bench.py.  It shares no code with the CUDA
library and never calls it.
"""
