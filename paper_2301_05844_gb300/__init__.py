"""GB300-native block belief propagation (blockBP) for 2D PEPS.

The compute path is a CUDA library (``libbbp.so``, built from ``csrc/`` for sm_103a)
behind the C ABI declared in ``include/bbp.h``; ``binding`` marshals arguments to it.
Importing this package loads nothing; ``binding.lib()`` opens the library and
raises if it is missing.
"""
