"""GB300-native SPH advection-dispersion hot path (Klapp et al., arXiv 2108.09488).

The compute path is the C-ABI library ``libade_sph.so`` (hand-written sm_103a CUDA kernels).
``paper_2108_09488_gb300.ade`` is its thin ctypes binding; ``inputs`` builds seeded workloads.
Importing this package does not load the library; ``ade`` loads it on first use and raises if it
is missing.
"""
__all__ = ["inputs"]
