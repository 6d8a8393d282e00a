"""The multi-process path on CPU: world size 2 over gloo. Each rank traces its photon-id shard
with the oracle, the shards' L are summed with an all-reduce, and the sum must equal the
single-process render; shard() must tile [0, N) for any world size."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_path):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1512_02110_gb300.shard import allreduce_sum_, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, p = synth.cfg_blobs16(n)
    off, cnt = shard(n, rank, world)
    r = oracle.render(sc, p.replace(n_photons=cnt, photon_offset=off, n_photons_total=n), nthreads=1)
    L = torch.from_numpy(r["L"])
    allreduce_sum_(L)
    if rank == 0:
        np.save(out_path, L.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_tiles_the_id_range():
    from paper_1512_02110_gb300.shard import shard
    for n in (0, 1, 7, 1000, 10**8 + 3):
        for world in (1, 2, 3, 8):
            ranges = [shard(n, r, world) for r in range(world)]
            assert sum(c for _, c in ranges) == n
            pos = 0
            for off, cnt in ranges:
                assert off == pos
                pos += cnt
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def test_two_rank_gloo_sum_equals_single_process(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    import torch.multiprocessing as mp

    import oracle
    import synth
    n = 30_001
    out = str(tmp_path / "L.npy")
    mp.spawn(_worker, args=(2, _free_port(), n, out), nprocs=2, join=True)
    sc, p = synth.cfg_blobs16(n)
    full = oracle.render(sc, p, nthreads=1)["L"]
    L = np.load(out)
    assert np.allclose(L, full, rtol=1e-12, atol=1e-300)
