"""FP64 CPU oracle of the ROKS plane-wave hot path.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  The CUDA library and its Python
binding never use it.
"""
