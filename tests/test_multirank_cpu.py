"""Host-side model of sharding the path over GPUs by detector, the paper's
data distribution (every process holds a subset of the samples and the
operators act collectively, the pointing operator's pixel sum reduced over
processes; Sec. III-A item 1, Sec. III-B): each rank owns whole detectors, so
no Toeplitz chunk crosses a rank, computes its partial P^T N^-1 P x and
P^T N^-1 d over its own samples, and one sum over ranks gives the full
operator.  World size 2 over gloo on the CPU, computed with the oracle; the
GPU build runs one replica per rank (one GPU per process, no data-path
collective)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system(noise_kind):
    import synth
    from oracle import gls
    e = synth.make_experiment(16, 6, 12_000, 4321)
    pt = synth.pointing(e, flag_frac=0.01)
    inv_var = 1.0 / e.sigma ** 2
    if noise_kind == "white":
        noise = gls.WhiteNoise(inv_var, e.det_offsets)
    else:
        coeffs = synth.toeplitz_band(e.sigma, 0.2, 1.0, 20.0, 4096, 48)
        noise = gls.ToeplitzNoise(coeffs, e.det_offsets, 4096, inv_var)
    return e, pt, gls.System(pt["pix"], pt["psi"], 3, e.npix, noise)


def _worker(rank, world, port, noise_kind, results):
    import torch.distributed as dist
    from oracle import gls
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        e, pt, S = _system(noise_kind)
        x = np.random.default_rng(7).normal(size=(e.npix, 3))
        d = np.random.default_rng(8).normal(size=e.nsamples)
        # this rank's detectors and their samples: the library's partition
        from paper_2501_16122_gb300.shard import detector_shard
        d0, d1, _ = detector_shard(e.det_offsets, rank, world)
        mine = list(range(d0, d1))
        off = np.asarray(e.det_offsets)
        idx = np.concatenate([np.arange(off[k], off[k + 1]) for k in mine])
        sub_off = np.concatenate([[0], np.cumsum([off[k + 1] - off[k] for k in mine])])
        if noise_kind == "white":
            noise = gls.WhiteNoise(np.asarray(S.noise.inv_var)[mine], sub_off)
        else:
            noise = gls.ToeplitzNoise(np.asarray(S.noise.coeffs)[mine], sub_off, S.noise.chunk_len,
                                      np.asarray(S.noise.white_inv_var)[mine])
        pe, v = S.pe[idx], S.v[idx]  # the global mask decides which rows are zero
        q = gls.apply_PT(pe, v, noise.apply(gls.apply_P(pe, v, x)), e.npix)
        dm = np.where(pe >= 0, d[idx], 0.0)
        b = gls.apply_PT(pe, v, noise.apply(dm), e.npix)
        t = torch.from_numpy(np.concatenate([q.ravel(), b.ravel()]))
        dist.all_reduce(t)
        if rank == 0:
            full_q, full_b = S.matvec(x), S.rhs(d)
            got = t.numpy()
            nq = full_q.size
            results.put((np.linalg.norm(got[:nq] - full_q.ravel()) / np.linalg.norm(full_q),
                         np.linalg.norm(got[nq:] - full_b.ravel()) / np.linalg.norm(full_b)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("noise_kind", ["white", "toeplitz"])
def test_detector_sharding_sums_to_the_full_operator(noise_kind):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, noise_kind, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    eq, eb = results.get(timeout=5)
    assert eq < 1e-13 and eb < 1e-13, (eq, eb)


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_detector_shard_partition(world):
    """Every detector belongs to exactly one rank, in order, each rank at
    least one, about as many samples each; the local offsets start at 0."""
    from paper_2501_16122_gb300.shard import detector_shard
    rng = np.random.default_rng(world)
    lens = rng.integers(1, 1000, 13)
    off = np.concatenate([[0], np.cumsum(lens)])
    prev = 0
    sizes = []
    for r in range(world):
        d0, d1, sub = detector_shard(off, r, world)
        assert d0 == prev and d1 > d0
        assert sub[0] == 0 and np.array_equal(sub, off[d0:d1 + 1] - off[d0])
        sizes.append(off[d1] - off[d0])
        prev = d1
    assert prev == 13
    assert max(sizes) <= off[-1] / world + lens.max()
    with pytest.raises(ValueError):
        detector_shard(off, 0, 14)
