"""GB300-native hierarchical-inverse EMT network solver.

The compute path is the native library libemt_hinv.so (CUDA for sm_103a plus C++ host code)
behind the C ABI in include/emt.h; ``paper_2105_10661_gb300._lib`` is its thin ctypes binding
and ``paper_2105_10661_gb300.buildlib`` compiles it. Importing the package does not load the
library; importing ``_lib`` does, and fails loudly if it has not been built.
"""
