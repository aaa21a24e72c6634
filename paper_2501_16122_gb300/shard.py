"""Host-side partition of a detector-sharded solve (paper Sec. III-A item 1:
every process owns a subset of the samples).  Pure Python: no library load."""
from __future__ import annotations

import numpy as np


def detector_shard(det_offsets, rank: int, world: int):
    """The detectors of one rank of a detector-sharded solve: contiguous
    blocks of whole detectors with about as many samples each, at least one
    detector a rank (world <= number of detectors).  Returns (first detector, end detector,
    this rank's det_offsets starting at 0)."""
    off = np.asarray(det_offsets, np.int64)
    ndet = off.size - 1
    if not (0 <= rank < world) or ndet < world:
        raise ValueError("bad rank or det_offsets, or more ranks than detectors")
    total = off[-1]
    # detector boundaries closest to rank * total / world
    cuts = [0] + [int(np.searchsorted(off, k * total / world, side="left")) for k in range(1, world)] + [ndet]
    for k in range(1, world):  # at least one detector per rank
        cuts[k] = min(max(cuts[k], cuts[k - 1] + 1), ndet - (world - k))
    d0, d1 = int(cuts[rank]), int(cuts[rank + 1])
    return d0, d1, off[d0:d1 + 1] - off[d0]
