"""GB300-native GLS map-making (the hot path of BrahMap, arXiv 2501.16122).

The computation lives in ``libbrahmap.so`` (hand-written CUDA for sm_103a,
C-ABI in ``include/brahmap.h``); ``_lib`` is its ctypes binding with the same
function names.  Build the library with :func:`build`.
"""
from __future__ import annotations

import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    from .nvcc_build import build as _build
    return _build(verbose_ptxas=verbose_ptxas, force=force)


def lib():
    """The loaded binding module (raises ImportError if the library was not built)."""
    from . import _lib
    return _lib
