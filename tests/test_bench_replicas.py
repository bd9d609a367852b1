"""The benchmark's multi-rank path on CPU (gloo, world size 2).

bench.py times every configuration through `timed_over_ranks`: warm-up, a
barrier and a synchronisation on both sides of exactly `steps` timed steps,
and the max over ranks.  Its strong-scaling split gives each rank the
tensors `replicas.shard_by_size` assigns it.  Here two gloo ranks drive that
same code with a CPU timer: the reported time is the slower rank's, every
tensor of the ResNet-18 set is run by exactly one rank, the per-rank results
(computed by the oracle) equal the single-process ones, and the reference arm
does its work on rank 0 only."""
import os
import socket
import time

import numpy as np
import torch.multiprocessing as mp

SIZES = [257, 1000, 33, 4096, 512, 77, 2048, 9]


class _CpuTimer:
    device = None

    def sync(self):
        pass

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        return 1e3 * (time.perf_counter() - self.t0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    from paper_2309_04909_gb300.replicas import shard_by_size
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # timing: rank 1's steps are slower; every rank must report rank 1's time
    calls = []

    def step():
        calls.append(1)
        time.sleep(0.002 if rank == 0 else 0.02)

    own, mx = bench.timed_over_ranks(step, 5, 3, world, _CpuTimer())
    # strong split of the tensors, computed by the oracle on each rank
    mine = shard_by_size(SIZES, world)[rank]
    P = O.params(64, 24, 0)
    outs = {}
    for t in mine:
        x = W.magnitude_bounded_ints(SIZES[t], 23, seed=t)
        s0, s1 = O.share(64, x.astype(np.uint64), 5, t)
        outs[t] = O.relu(P, s0, s1, 5, 100 + t)
    gathered = [None] * world
    dist.all_gather_object(gathered, (own, mx, len(calls), outs))
    # the reference arm: ranks other than 0 return at once without work
    t0 = time.perf_counter()
    if rank != 0:
        ref = bench.run_reference(None)
        assert ref is None
    ref_s = time.perf_counter() - t0
    if rank == 0:
        np.save(os.path.join(out_dir, "timing.npy"),
                np.array([[g[0], g[1], g[2]] for g in gathered]))
        merged = {}
        for g in gathered:
            assert not set(merged) & set(g[3])
            merged.update(g[3])
        for t, (o0, o1) in merged.items():
            np.save(os.path.join(out_dir, f"t{t}.npy"), np.stack([o0, o1]))
    else:
        np.save(os.path.join(out_dir, "ref_rank1.npy"), np.array([ref_s]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_timing_and_split_two_gloo_ranks(tmp_path):
    import oracle as O
    from paper_2309_04909_gb300 import workloads as W
    O.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    tm = np.load(tmp_path / "timing.npy")
    # 3 warm-up + 5 timed steps on every rank
    assert (tm[:, 2] == 8).all()
    # both ranks report the max, which is rank 1's own time (>= 5 x 20 ms)
    assert tm[0, 1] == tm[1, 1] == max(tm[0, 0], tm[1, 0])
    assert tm[1, 0] >= 100.0 and tm[0, 1] >= tm[1, 0]
    assert float(np.load(tmp_path / "ref_rank1.npy")[0]) < 1.0
    P = O.params(64, 24, 0)
    for t, n in enumerate(SIZES):
        x = W.magnitude_bounded_ints(n, 23, seed=t)
        s0, s1 = O.share(64, x.astype(np.uint64), 5, t)
        o0, o1 = O.relu(P, s0, s1, 5, 100 + t)
        got = np.load(tmp_path / f"t{t}.npy")
        assert np.array_equal(got[0], o0) and np.array_equal(got[1], o1)


def test_strong_split_covers_the_resnet18_set():
    from paper_2309_04909_gb300 import workloads as W
    from paper_2309_04909_gb300.replicas import shard_by_size
    sizes = (W.RESNET18_224_LAYERS * 32) * 2
    for world in (2, 4, 8):
        shards = shard_by_size(sizes, world)
        assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)
