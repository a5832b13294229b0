"""Multi-rank path on CPU: world_size 2 over gloo.

Each rank evaluates its slice of a batch of cells and pairs with the FP64
oracle (standing in for its GPU); the slices, gathered only to check them,
must equal the single-rank batch exactly.  The data path itself has no
collective.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2112_02695_gb300.sharding import inputs_used, shard_pairs, shard_range

CFG = dict(N=8, d=3, L=8.0, R=8.0, gamma=1.0, n_rho=3, M=6)


def test_shard_range_covers_exactly_once():
    for n in (0, 1, 5, 256, 257, 512):
        for world in (1, 2, 3, 8):
            seen = [e for r in range(world) for e in shard_range(n, world, r)]
            assert seen == list(range(n))
            sizes = [len(shard_range(n, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import collision as C
    from paper_2112_02695_gb300 import workloads as W
    prob = C.Problem(**CFG)
    fields = W.random_fields(8, 3, 8.0, 5, seed=77)
    pairs = [(j, l) for j in range(3) for l in range(3)] + [(x, x) for x in range(3, 5)]
    mine, rng = shard_pairs(pairs, world, rank)
    used = inputs_used(mine)
    local = {g: i for i, g in enumerate(used)}
    Q = C.collide_fields(prob, fields[used], [(local[a], local[b]) for a, b in mine])
    gathered = [None] * world
    dist.all_gather_object(gathered, (list(rng), Q))        # verification only
    if rank == 0:
        idx = [e for r, _ in gathered for e in r]
        allq = np.concatenate([q for _, q in gathered])
        np.save(os.path.join(out_dir, "sharded.npy"), allq[np.argsort(idx)])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_single_rank(tmp_path):
    from oracle import collision as C
    from paper_2112_02695_gb300 import workloads as W
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "sharded.npy")
    prob = C.Problem(**CFG)
    fields = W.random_fields(8, 3, 8.0, 5, seed=77)
    pairs = [(j, l) for j in range(3) for l in range(3)] + [(x, x) for x in range(3, 5)]
    ref = C.collide_fields(prob, fields, pairs)
    assert np.array_equal(got, ref) or np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
