"""GB300-native Lloyd k-means with MTI pruning (knor, arXiv 1606.08905).

The compute path is a C-ABI shared library, ``libknor.so``, built from the CUDA
sources in ``csrc/`` for sm_103a; ``knor`` is its thin ctypes binding and
``synth`` draws the seeded synthetic workloads.  Importing this package loads
nothing; ``knor.load()`` (called by every binding entry point) loads the
library and raises if it has not been built.
"""
__all__ = ["knor", "synth", "build"]
