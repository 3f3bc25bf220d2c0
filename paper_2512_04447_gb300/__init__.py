"""GB300-native (sm_103a) real-space Kohn-Sham LOBPCG path.

The compute lives in ``librsdft.so`` (CUDA, built in-tree by ``build.py``);
``rsdft`` is its Python binding.  Nothing here falls back to the CPU.
"""
from . import rsdft  # noqa: F401
