"""polyrx: GB300-native reactive coarse-grained MD (de Buyl & Nies, arXiv:1409.7498).

The compute path is libpolyrx.so (hand-written CUDA for sm_103a) behind the C
ABI of include/polyrx.h; ``polyrx`` is its ctypes binding and ``build``
compiles it in-tree.  Importing this package loads nothing; the binding
loads the library on first use and raises if it is missing.
"""
