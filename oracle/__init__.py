"""FP64 CPU oracle for GLS map-making — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct numpy implementations of what the CUDA library
computes: HEALPix RING ang2pix/pix2ang (``healpix``), the pointing operator,
white and banded-Toeplitz inverse noise, the block-diagonal preconditioner
with its hit/condition mask, PCG, and a dense Cholesky solve for tiny
problems (``gls``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg import this package.  It shares no code with the CUDA library
and never imports it; the library never imports this package.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, textbook pixel centres,
round trips, brute force, a dense direct solve, invariants).  No function is
"parity unpinned".
"""
from . import healpix, gls  # noqa: F401
from .healpix import ang2pix_ring, pix2ang_ring, nside2npix  # noqa: F401
from .gls import (System, WhiteNoise, ToeplitzNoise, pcg, gls_map, dense_gls,  # noqa: F401
                  pointing_weights, block_matrices, block_condition, pixel_mask, rel_err)
