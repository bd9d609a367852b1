"""Multi-rank layout on CPU (gloo, world size 2): the shards cover every
tensor exactly once, each rank's results (computed here by the oracle) equal
the single-process results, and the timing reduction takes the max."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2309_04909_gb300.replicas import max_over_ranks, rank_seed, shard_by_size


def test_shard_by_size_balanced_and_complete():
    rng = np.random.default_rng(0)
    sizes = [int(x) for x in rng.integers(1, 100_000, size=1664)]
    for world in (1, 2, 4, 8):
        shards = shard_by_size(sizes, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)


def test_rank_seeds_distinct():
    assert len({rank_seed(7, r) for r in range(64)}) == 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_dir):
    import torch.distributed as dist
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [257, 1000, 33, 4096, 512, 77, 2048, 9]
    mine = shard_by_size(sizes, world)[rank]
    P = O.params(64, 24, 0)
    outs = {}
    for t in mine:
        x = W.magnitude_bounded_ints(sizes[t], 23, seed=t)
        s0, s1 = O.share(64, x.astype(np.uint64), 5, t)
        o0, o1 = O.relu(P, s0, s1, 5, 100 + t)
        outs[t] = (o0, o1)
    gathered = [None] * world
    dist.all_gather_object(gathered, outs)
    mx = max_over_ranks(float(rank + 1))
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        np.save(os.path.join(result_dir, "ok.npy"),
                np.array([len(merged) == len(sizes), mx == float(world)]))
        for t, (o0, o1) in merged.items():
            np.save(os.path.join(result_dir, f"t{t}.npy"), np.stack([o0, o1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process(tmp_path):
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    O.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    ok = np.load(tmp_path / "ok.npy")
    assert ok.all()
    P = O.params(64, 24, 0)
    for t, n in enumerate([257, 1000, 33, 4096, 512, 77, 2048, 9]):
        x = W.magnitude_bounded_ints(n, 23, seed=t)
        s0, s1 = O.share(64, x.astype(np.uint64), 5, t)
        o0, o1 = O.relu(P, s0, s1, 5, 100 + t)
        got = np.load(tmp_path / f"t{t}.npy")
        assert np.array_equal(got[0], o0) and np.array_equal(got[1], o1)
