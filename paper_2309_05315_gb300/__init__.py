"""GB300 (sm_103a) implementation of the Method of Averaged Marginals.

The compute path is libmam.so (CUDA kernels behind the C ABI of
include/mam.h); ``Mam`` is its Python binding and ``torch_api`` adds a
``torch.autograd.Function`` on top.  Build the library with
``paper_2309_05315_gb300.build.build()``.
"""
from ._capi import MamError, lib  # noqa: F401
from .mam import Mam  # noqa: F401
