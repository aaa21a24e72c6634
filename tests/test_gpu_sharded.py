"""The detector-sharded solve through the library (the paper's data
distribution, Sec. III-A item 1, with the pointing operator's partial map
summed over the processes, Sec. III-B): two ranks, each a process with its
own library context on the one GPU, holding half of the detectors and summing
per-pixel partial results with gloo on the host (no kernel of one rank waits
for the other's).  What rank 0 computed must match the single-process solve
of all detectors to rounding (the partial sums are added in another order)
and the FP64 oracle within the usual bounds; hit counts and the mask are
exact.  White noise (with the TOD carried through the sort) and a 64-lag
Toeplitz N^-1."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from oracle import gls

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import shard_worker  # noqa: E402


@pytest.fixture(scope="module")
def L():
    import paper_2501_16122_gb300 as pkg
    pkg.build()
    from paper_2501_16122_gb300 import _lib
    return _lib


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def run_sharded(case, world, tmp_path):
    port = _free_port()
    out = str(tmp_path / f"{case}_{world}.npz")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "shard_worker.py"), str(r), str(world), str(port),
                               case, out], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for r in range(world)]
    logs = []
    for pr in procs:
        try:
            logs.append(pr.communicate(timeout=600)[0])
        except subprocess.TimeoutExpired:
            pr.kill()
            logs.append(pr.communicate()[0])
    for pr, log in zip(procs, logs):
        assert pr.returncode == 0, log[-3000:]
    return dict(np.load(out))


@pytest.mark.parametrize("case", ["white", "toeplitz"])
def test_sharded_solve_matches_single_process_and_oracle(L, case, tmp_path):
    inp = shard_worker.case_inputs(case)
    e = inp["e"]
    ctx = L.bm_context_create(0)
    try:
        single = shard_worker.solve(L, ctx, inp, 0, e.ndet, e.det_offsets)
    finally:
        L.bm_context_destroy(ctx)
    shard = run_sharded(case, 2, tmp_path)

    # integers: exact
    assert np.array_equal(shard["hits"], single["hits"])
    assert np.array_equal(shard["mask"], single["mask"])
    # per-pixel sums of two partials: the same values to rounding (FP64
    # operators), or to the FP32 products' rounding (the mixed operator,
    # whose FP32 groups of samples differ with the split)
    for k, tol in (("q_fp64", 1e-12), ("b", 1e-12), ("pt_y", 1e-12), ("q_mixed", 2e-6)):
        assert rel(shard[k], single[k]) < tol, (k, rel(shard[k], single[k]))
    mask = single["mask"].astype(bool)
    keep = np.repeat(~mask, 3)
    for k in ("map_fp64", "map_mixed") + (("map_carried",) if case == "white" else ()):
        assert np.array_equal(np.isnan(shard[k]), np.isnan(single[k])), k
        assert rel(shard[k][keep], single[k][keep]) < 1e-8, (k, rel(shard[k][keep], single[k][keep]))

    # the oracle's GLS map of all detectors
    if case == "white":
        noise = gls.WhiteNoise(1.0 / e.sigma ** 2, e.det_offsets)
        S = gls.System(inp["pix"], None, 3, e.npix, noise, trig=(inp["c32"], inp["s32"]))
    else:
        noise = gls.ToeplitzNoise(inp["coeffs"], e.det_offsets, inp["chunk"], 1.0 / e.sigma ** 2)
        S = gls.System(inp["pix"], inp["psi"], 3, e.npix, noise)
    assert np.array_equal(S.mask, mask)
    ref, _ = gls.gls_map(S, np.asarray(inp["tod"], np.float64), tol=1e-13)
    for k, tol in (("map_fp64", 1e-10), ("map_mixed", 1e-6)):
        err = gls.rel_err(shard[k].reshape(e.npix, 3), ref, S.mask)
        assert max(err.values()) < tol, (k, err)
    x = np.random.default_rng(9).normal(size=(e.npix, 3))
    assert rel(shard["q_fp64"], S.matvec(x).ravel()) < 1e-12
