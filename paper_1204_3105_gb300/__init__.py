"""GB300-native 2D fast multipole method over quadtree, septree and
triangle-quadtree tilings (Luo & Duraiswami, arXiv:1204.3105).

The compute path is the C-ABI library ``libfmm2d.so`` built from ``csrc/``
for sm_103a; ``paper_1204_3105_gb300.fmm2d`` is its thin ctypes binding.
Importing this package does not load the library; ``fmm2d.lib()`` does, and
raises if it has not been built.
"""
__all__ = ["fmm2d", "inputs"]
