"""Multi-rank query sharding on CPU (torch.distributed gloo, world size 2): the shards,
evaluated with their global Philox ids, gather to the single-process result exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2407_06107_b300.sharding import shard, weak_id_base


def test_shard_partition():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == n
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    assert weak_id_base(3, 1 << 24) == 3 << 24


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import stf_synth as synth
    m = synth.material_rgba8(32, 4, octaves=3, base=2)
    tex = oracle.Texture(m.albedo_rough, m.normal)
    q = synth.queries_uniform(301, 5, res=32, lod_range=4.0)
    b, c = shard(q.n, rank, world)
    idx = np.arange(b, b + c)
    r = oracle.filter_shade(tex, q.subset(idx), "mitchell", "stochastic", spp=3, seed=7, ids=idx, nthreads=1)
    parts = [None] * world
    dist.all_gather_object(parts, r.rgb)
    # the bench's max-over-ranks timing reduction
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(out_path, np.concatenate(parts))
        assert float(t) == world
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process(tmp_path):
    out = str(tmp_path / "gathered.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    import oracle
    import stf_synth as synth
    m = synth.material_rgba8(32, 4, octaves=3, base=2)
    q = synth.queries_uniform(301, 5, res=32, lod_range=4.0)
    whole = oracle.filter_shade(oracle.Texture(m.albedo_rough, m.normal), q, "mitchell", "stochastic", spp=3,
                                seed=7, nthreads=1)
    assert np.array_equal(np.load(out), whole.rgb)
