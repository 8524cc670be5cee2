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


# ----------------------------------------------------------------- data-parallel training
def _dp_problem():
    import oracle
    import stf_synth as synth
    grids, R0 = (8, 4, 2, 1), 16
    lat, mlp = synth.ntc_init(grids, 41)
    mlp[2048:2112] = 0.05
    tg = synth.ntc_targets(synth.material_rgba8(R0, 42, octaves=3, base=2, mips=False), 43)
    return oracle, grids, R0, lat, mlp, tg


class _OracleReplica:
    """One replica of the learned form on the FP64 oracle: FP32 master parameters, gradients
    of a share of each step's batch normalised by the whole batch, Adam."""

    def __init__(self, batch, seed=5, lr=(1e-2, 5e-3)):
        self.oracle, self.grids, self.R0, lat, mlp, self.tg = _dp_problem()
        self.p = np.concatenate([g.ravel() for g in lat] + [mlp]).astype(np.float64)
        self.nl = sum(g.size for g in lat)
        self.m, self.v = np.zeros_like(self.p), np.zeros_like(self.p)
        self.g = np.zeros_like(self.p)
        self.batch, self.seed, self.lr = batch, seed, lr

    def params32(self):
        p = self.p.astype(np.float32)
        lat, o = [], 0
        for r in self.grids:
            lat.append(p[o:o + r * r * 8].reshape(r, r, 8))
            o += r * r * 8
        return lat, p[self.nl:]

    def grad(self, k, first, count):
        self.g[:] = 0.0
        if count == 0:
            return
        ix, iy = self.oracle.ntc_sample_texels(k, self.batch, self.seed, self.R0)
        lat, mlp = self.params32()
        _, gm, gl = self.oracle.ntc_loss_grad(self.R0, lat, mlp, self.tg, ix[first:first + count],
                                              iy[first:first + count], round_bf16=True)
        # the oracle normalises by its own sample count; the share's part of the batch mean
        # (exact, since the FP64 backward is linear in that normalisation)
        self.g[:self.nl] = gl * (count / self.batch)
        self.g[self.nl:] = gm * (count / self.batch)

    def adam(self, k):
        for sl, lr in ((slice(0, self.nl), self.lr[0]), (slice(self.nl, None), self.lr[1])):
            p, m, v = self.p[sl].copy(), self.m[sl].copy(), self.v[sl].copy()
            self.oracle.adam(p, self.g[sl].copy(), m, v, k + 1, lr)
            self.p[sl], self.m[sl], self.v[sl] = p, m, v


def _dp_worker(rank, world, port, out_path, steps, batch):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2407_06107_b300.sharding import dp_train
    rep = _OracleReplica(batch)
    calls = []

    def allreduce():
        t = torch.from_numpy(rep.g)
        dist.all_reduce(t)            # in place on the replica's gradient array
        calls.append(1)
    dp_train(steps, batch, rank, world, rep.grad, allreduce, rep.adam)
    assert len(calls) == steps
    parts = [None] * world
    dist.all_gather_object(parts, rep.p)
    if rank == 0:
        np.save(out_path, np.stack(parts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_data_parallel_training_matches_one_process(tmp_path):
    # 3 optimiser steps of a 301-sample batch (shards 151 + 150): the replicas stay
    # identical, and equal the single-process run up to the order of the gradient sums
    steps, batch = 3, 301
    out = str(tmp_path / "dp.npy")
    mp.spawn(_dp_worker, args=(2, _free_port(), out, steps, batch), nprocs=2, join=True)
    reps = np.load(out)
    assert np.array_equal(reps[0], reps[1])
    from paper_2407_06107_b300.sharding import dp_train
    one = _OracleReplica(batch)
    dp_train(steps, batch, 0, 1, one.grad, lambda: None, one.adam)
    np.testing.assert_allclose(reps[0], one.p, rtol=1e-6, atol=1e-9)
    # the run moved the parameters (the comparison is not vacuous)
    assert np.abs(one.p - _OracleReplica(batch).p).max() > 1e-3


def test_dp_train_calls_one_collective_per_step():
    from paper_2407_06107_b300.sharding import dp_train
    log = []
    dp_train(4, 10, 1, 3, lambda k, f, c: log.append(("g", k, f, c)), lambda: log.append(("r",)),
             lambda k: log.append(("a", k)))
    assert log[:3] == [("g", 0, 4, 3), ("r",), ("a", 0)] and len(log) == 12
    log.clear()
    dp_train(2, 10, 0, 1, lambda k, f, c: log.append(("g", k, f, c)), lambda: log.append(("r",)),
             lambda k: log.append(("a", k)))
    assert ("r",) not in log and log[0] == ("g", 0, 0, 10)


def _dp_leave_worker(rank, world, port, out_dir):
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    from paper_2407_06107_b300.sharding import dp_train
    g = np.zeros(64)

    def grad(k, first, count):
        g[:] = k + rank

    def allreduce():
        dist.all_reduce(torch.from_numpy(g))

    def adam(k):
        if rank == 1 and k == 1:
            os._exit(0)          # this rank leaves between steps, with no collective in flight
    t0 = time.time()
    try:
        dp_train(5, 10, rank, world, grad, allreduce, adam)
        result = "finished"
    except Exception:            # the surviving rank's next collective fails (closed peer / timeout)
        result = "error"
    with open(os.path.join(out_dir, f"rank{rank}"), "w") as f:
        f.write(f"{result} {time.time() - t0:.3f}")
    os._exit(0)                  # the group cannot be torn down without its peer


@pytest.mark.timeout(180)
def test_rank_leaving_between_steps_ends_the_others_next_collective(tmp_path):
    # failure detection on the host: when one data-parallel rank exits after step 1, the other
    # learns of it at step 2's all-reduce, which raises within the process group's timeout
    # instead of hanging
    mp.spawn(_dp_leave_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    result, secs = open(tmp_path / "rank0").read().split()
    assert result == "error" and float(secs) < 60.0
    assert not (tmp_path / "rank1").exists()
