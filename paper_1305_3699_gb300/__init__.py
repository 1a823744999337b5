"""GB300-native RNS modular exponentiation (the MR-MOD layer of "Secrets from the GPU").

The compute path lives in libmrmod.so (hand-written CUDA for sm_103a behind the
C ABI of include/mr.h); ``paper_1305_3699_gb300.mr`` is its ctypes binding.
Importing the binding raises ImportError when the library is not built.
"""

__all__ = ["mr"]
