"""GB300-native matrix-free hp-DG (SIPG) elliptic operator and multigrid solver.

The compute path is the CUDA library `libdgell.so` (built from csrc/) behind
the C ABI declared in include/dgell.h.  `paper_1907_01572_gb300.dgell` is the
thin ctypes binding; `paper_1907_01572_gb300.inputs` holds the seeded
synthetic workload generators.
"""
