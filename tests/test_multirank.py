"""The multi-rank path on CPU: world size 2 over gloo.  Each rank runs its
shard of walk indices (the oracle stands in for the GPU arm here); the
shards reproduce the single-process batch, and the step time is the maximum
over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2107_11983_gb300.shard import strong_shard, weak_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import oracle
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = synth.rmat(9, seed=2)
    src = synth.vertex_sources(g.nv)
    # strong split of one batch
    lo, hi = strong_shard(src.shape[0], rank, world)
    res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src[lo:hi], 15, 4, n2v_p=0.5, n2v_q=2.0, walk_offset=lo)
    assert res.status == 0
    np.save(os.path.join(out_dir, f"strong{rank}.npy"), res.paths)
    np.save(os.path.join(out_dir, f"strong_len{rank}.npy"), res.lengths)
    # weak split: every rank its own batch of the same size
    off = weak_shard(src.shape[0], rank)
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, src, 10, 4, walk_offset=off)
    np.save(os.path.join(out_dir, f"weak{rank}.npy"), res.paths)
    # max-over-ranks timing as the bench reduces it
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    assert t.item() == float(world)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_reproduce_single_process(tmp_path):
    import oracle
    import synth

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    g = synth.rmat(9, seed=2)
    src = synth.vertex_sources(g.nv)
    full = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, 15, 4, n2v_p=0.5, n2v_q=2.0)
    paths = np.concatenate([np.load(tmp_path / f"strong{r}.npy") for r in range(world)])
    lens = np.concatenate([np.load(tmp_path / f"strong_len{r}.npy") for r in range(world)])
    assert np.array_equal(lens, full.lengths)
    mask = np.arange(16)[None, :] < lens[:, None]
    assert np.array_equal(paths[mask], full.paths[mask])
    both = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, np.concatenate([src, src]), 10, 4)
    weak = np.concatenate([np.load(tmp_path / f"weak{r}.npy") for r in range(world)])
    m = np.arange(11)[None, :] < both.lengths[:, None]
    assert np.array_equal(weak[m], both.paths[m])


@pytest.mark.parametrize("n,world", [(0, 1), (10, 3), (7, 7), (5, 8), (1000003, 4)])
def test_strong_shard_partitions(n, world):
    ranges = [strong_shard(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and b >= a
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1
