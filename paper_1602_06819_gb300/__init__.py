"""Online k-nn graph building on one GB300 (Debatty, Michiardi, Mees, KDD'16).

The compute path is the CUDA library ``libknn_graph.so`` behind the C ABI in
``include/knn_graph.h``; :mod:`.knn` is its thin ctypes binding and
:mod:`.inputs` the seeded synthetic data.  Importing this package loads
nothing; importing :mod:`.knn` loads the library and fails loudly if it is
missing.
"""

__all__ = ["inputs", "knn"]
