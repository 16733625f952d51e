"""Pixel-sharded reconstruction on CPU (Sec. IV: G(k, K) and the trotter sum
of Eq. 3 are per detector pixel k): two gloo ranks each take the pixel range
the library assigns to their shard (eer4d_shard_range, host code), form the
oracle's share of the spectrum over their bright-field pixels and of the
Gbar0 sums, add the shares with the package's all-reduce helper, and form the
image.  It equals the oracle's unsharded phase to rounding.  No GPU: the
CUDA side of the same path is tested on one GPU in test_gpu_shards.py."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

AB = (60.0, 10.0, -20.0, 5.0e3, 0.25)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    import oracle as orc
    w = synth.workload(1, scan_ny=16, scan_nx=24)
    geom = synth.geometry(w)
    idx, off = synth.generate(w).numpy()
    G = orc.g_function(orc.densify(idx, off, geom), geom)
    return geom, G


def _share(geom, G, rank, world):
    import oracle as orc
    from paper_2104_06336_gb300.buildlib import build
    from paper_2104_06336_gb300 import _lib
    build()
    pt = orc.pixel_table(geom)
    b, e = _lib.eer4d_shard_range(pt["P"], rank, world)
    pix = np.arange(b, e)
    S, _ = orc.ssb_spectrum(G[pix], geom, AB, pixels=pix)
    bf = pix[pt["bf"][pix]]
    g0 = np.array([G[bf, 0, 0].real.sum(), float(len(bf))])
    return torch.from_numpy(S), torch.from_numpy(g0)


def _rank(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2104_06336_gb300.sharding import allreduce_partials
        geom, G = _case()
        S, g0 = _share(geom, G, rank, world)
        allreduce_partials(S, g0)
        NR = geom["scan_ny"] * geom["scan_nx"]
        phi = NR / (float(g0[0]) / float(g0[1])) * np.fft.ifft2(S.numpy()).imag
        q.put((rank, phi, g0.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_shares_add_up_to_the_whole(world):
    import oracle as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    geom, G = _case()
    phi, _ = orc.ssb_phase(G, geom, AB, "none")
    pt = orc.pixel_table(geom)
    for rank, ph, g0 in res:
        assert g0[1] == pt["bf"].sum()
        assert np.abs(ph - phi).max() <= 1e-10 * np.abs(phi).max(), rank


def test_shard_ranges_partition_the_pixels():
    """Host code only: the shards' ranges tile [0, P) without gaps or overlap,
    differ in size by at most one pixel, and bad arguments are refused."""
    from paper_2104_06336_gb300.buildlib import build
    from paper_2104_06336_gb300 import _lib
    build()
    for P in (1, 7, 553, 1245, 7209):
        for n in (1, 2, 3, 8, 64):
            if n > P:
                continue
            r = [_lib.eer4d_shard_range(P, s, n) for s in range(n)]
            assert r[0][0] == 0 and r[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [e - b for b, e in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    for bad in ((0, 0, 1), (10, 2, 2), (10, -1, 2), (10, 0, 65), (10, 0, 0)):
        with pytest.raises(_lib.Eer4dError):
            _lib.eer4d_shard_range(*bad)
