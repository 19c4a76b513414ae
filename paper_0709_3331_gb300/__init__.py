"""GB300-native TREE method for two-component ultracold plasmas (arXiv 0709.3331).

The compute path is ``libucp.so`` (CUDA, sm_103a) behind the C ABI of
``include/ucp.h``; :mod:`.ucp` is its Python binding and :mod:`.inputs` the
seeded synthetic cloud generator.
"""
from .ucp import (UCP_ELECTRON, UCP_FP32C, UCP_FP64, UCP_ION, Context,  # noqa: F401
                  UcpError, lib)
