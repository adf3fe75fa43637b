"""GB300-native template-matching orientation mapping (indexing hot path).

The compute path lives in the CUDA library ``libtmgb.so`` (built from ``csrc/``);
``tmgb`` is its thin ctypes binding.  Importing this package loads nothing.
"""
