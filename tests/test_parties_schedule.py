"""The message schedule of the three-process party mapping on CPU (gloo,
world size 3): each party's stages receive exactly the messages Alg. drelu /
Alg. relu send them, from the right sender, and every message is counted per
direction.  The stages here are stand-ins that write known values; the GPU
test of the real stages is in test_gpu_parties.py."""
import os
import time
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

N = 1000
WORDS = 3 * N + 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _stages():
    from paper_2309_04909_gb300.parties import Stages

    def buffers(prm, n):
        return {"w": torch.zeros(WORDS, dtype=torch.int32),
                **{k: torch.zeros(n, dtype=torch.int64) for k in ("open", "reply", "pre_c1",
                                                                 "out")}}

    def local(me, prm, relu, share, tid, buf):
        assert int(share[0]) == 10 + me
        buf["w"].fill_(100 + me)
        if relu:
            buf["open"].fill_(200 + me)
        return buf["w"], (buf["open"] if relu else None)

    def helper(prm, relu, tid, w0, w1, buf):
        assert (w0 == 100).all() and (w1 == 101).all()
        buf["reply"].fill_(300)
        buf["pre_c1"].fill_(400)
        return buf["reply"], (buf["pre_c1"] if relu else None)

    def finish(me, prm, relu, share, tid, reply, open0, open1, pre_c1, buf):
        out = buf["out"]
        for j, t in enumerate((reply, open0, open1, pre_c1)):
            out[j] = -1 if t is None else int(t[0])
        return out

    return Stages(local, helper, finish, buffers)


def _worker(rank, port, out_dir):
    import torch.distributed as dist
    from paper_2309_04909_gb300.parties import PartyProcess, Transport
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=3)
    res = {}
    for relu in (False, True):
        tr = Transport(torch.device("cpu"), direct=False)
        pp = PartyProcess(rank, _stages(), tr, clock=time.perf_counter)
        share = None if rank == 2 else torch.full((N,), 10 + rank, dtype=torch.int64)
        out = pp.run(None, relu, share, N, 7)
        res[relu] = (None if out is None else out[:4].clone().numpy(), dict(tr.sent),
                     dict(pp.timing))
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([res], dtype=object),
            allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_three_party_schedule_gloo(tmp_path):
    mp.start_processes(_worker, args=(_free_port(), str(tmp_path)), nprocs=3, join=True,
                       start_method="spawn")
    r = [np.load(tmp_path / f"r{k}.npy", allow_pickle=True)[0] for k in range(3)]
    wb, lb = WORDS * 4, N * 8
    # DReLU: P0 needs no message back, P1 gets [DReLU']_1 from P2
    assert list(r[0][False][0]) == [-1, -1, -1, -1]
    assert list(r[1][False][0]) == [300, -1, -1, -1]
    assert r[0][False][1] == {(0, 2): wb}
    assert r[1][False][1] == {(1, 2): wb}
    assert r[2][False][1] == {(2, 1): lb}
    # ReLU: openings exchanged, e to both, [c]_1 to P1 only
    assert list(r[0][True][0]) == [300, 200, 201, -1]
    assert list(r[1][True][0]) == [300, 200, 201, 400]
    assert r[0][True][1] == {(0, 2): wb, (0, 1): lb}
    assert r[1][True][1] == {(1, 2): wb, (1, 0): lb}
    assert r[2][True][1] == {(2, 0): lb, (2, 1): 2 * lb}
    assert r[2][True][0] is None
    # with a clock, each party's time splits into its stages and its messages
    for k in range(3):
        for relu in (False, True):
            tm = r[k][relu][2]
            assert set(tm) == {"compute", "transport"}
            assert tm["compute"] >= 0 and tm["transport"] > 0
