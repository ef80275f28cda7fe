"""GB300-native graph-guided k-means (GK-means, arXiv 1705.01813).

The compute path is the CUDA library ``libgkm.so`` built from ``csrc/``; the
Python binding in :mod:`paper_1705_01813_gb300.gkm` only marshals arguments to
its C entry points.  Nothing is imported eagerly, so that the synthetic-input
module :mod:`paper_1705_01813_gb300.datagen` loads without the library.
"""
__all__ = ["gkm", "datagen"]
