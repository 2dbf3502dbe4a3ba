"""GB300-native Fast CoveringLSH (fcLSH) hot path.

Exact Hamming-space r-near-neighbour reporting after Pham & Pagh, "Scalability
and Total Recall with Fast CoveringLSH" (arXiv 1602.02620): every point is hashed
into all covering-LSH keys by Algorithm 2 (sketch + fast Hadamard transform),
the keys are grouped into per-table bucket directories, and queries probe the
buckets, remove duplicate candidates and verify them by popcount distance
(Strategy 2).  All of it runs in the CUDA library ``libfclsh.so`` behind the C
ABI declared in ``include/fclsh.h``; :mod:`.fclsh` is its thin ctypes binding.

Importing this package loads nothing; the library is opened on first use and
fails loudly if it has not been built.
"""
__all__ = ["fclsh", "workloads"]
