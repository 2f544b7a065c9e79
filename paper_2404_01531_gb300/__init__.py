"""GB300-native library for the GRFFE DG-FD hybrid scheme of arXiv:2404.01531.

The compute path is the CUDA library libffe.so (csrc/, C ABI in include/ffe.h);
`ffe` is its ctypes binding.  Importing the package does not load the library;
`ffe.load()` does and raises if it is missing.
"""
from . import ffe  # noqa: F401
