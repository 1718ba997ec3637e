"""GB300-native inverse-overlap factorization Z Z^T = S^{-1} (arXiv:2404.19163).

The compute path is libzfact.so (CUDA, sm_103a) behind the C ABI in
include/zfact.h; ``zfact`` is its ctypes binding and ``synth`` the seeded
input generators."""
from .zfact import (Context, ZfactError, load, make_opts, PRECISION, REFINE_MODE,  # noqa: F401
                    EXPORTED, MLP_NPARAMS, LIB_PATH)
