"""GB300-native nested shift-invert MINRES for the periodic random-field
Heisenberg chain (Kutsuzawa & Todo, arXiv:2203.09732).

Import is lightweight: the CUDA library is loaded on first use by
``paper_2203_09732_gb300.hs`` (the ctypes binding of the C ABI in
``include/hs.h``). ``paper_2203_09732_gb300.inputs`` holds the seeded synthetic
input generators shared by tests and the benchmark.
"""
