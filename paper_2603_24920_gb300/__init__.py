"""GB300-native (sm_103a) DET-LSH hot path: C-ABI library + thin binding.

The CUDA library libdetlsh.so (csrc/, declared in include/detlsh.h) does all
of the work; ``detlsh`` marshals arguments to it.
"""
from . import detlsh  # noqa: F401
