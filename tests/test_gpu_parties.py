"""Party-separated DReLU/ReLU on the GPU: the three launches (P0/P1 local
work, P2, P0/P1 finish) exchange every message through device buffers and
give the fused kernel's outputs and the oracle's messages, bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import BicoptorError, Context, Params, workloads as W
from tests._util import masked, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED = 0x9A27_1E5


def padded_groups(n: int) -> int:
    """Groups of 32 elements in a packed buffer: whole CTAs of 8 groups."""
    return -(-n // 256) * 8


def unpack_w(words: np.ndarray, lx: int, n: int) -> np.ndarray:
    """Inverse of the packed message layout (group-major: group g, slot k at
    words (g L + k) B): (n, lx+1) values."""
    B, L, G = lx + 1, lx + 1, padded_groups(n)
    w = words.view(np.uint32).astype(np.uint64).reshape(G, L, B).transpose(1, 0, 2)
    bits = np.zeros((L, G, 32 * B), dtype=np.uint8)
    for b in range(32):
        bits[:, :, b::32] = ((w >> np.uint64(b)) & np.uint64(1)).astype(np.uint8)
    vals = np.zeros((L, G, 32), dtype=np.uint64)
    for b in range(B):
        vals |= bits[:, :, np.arange(32) * B + b].astype(np.uint64) << np.uint64(b)
    return vals.reshape(L, G * 32)[:, :n].T


CASES = [(64, 24, 0, 23, 10_007), (32, 9, 14, 22, 4_099), (32, 14, 4, 17, 3_000),
         (64, 7, 0, 6, 64), (64, 31, 2, 32, 1_001), (16, 5, 2, 6, 33),
         # one element; one full group; a CTA one short of / exactly / one past 256
         (64, 24, 0, 23, 1), (64, 24, 0, 23, 32), (64, 24, 0, 23, 255), (64, 24, 0, 23, 256),
         (32, 14, 4, 17, 257)]


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", CASES)
def test_parties_match_fused_and_oracle(op, ring, lx, c, mag, n):
    ctx = Context(SEED)
    x = W.magnitude_bounded_ints(n, mag, seed=n + lx)
    s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 5)
    prm = Params(ring, lx, c)
    fused = ctx.drelu if op == "drelu" else ctx.relu
    parties = ctx.drelu_parties if op == "drelu" else ctx.relu_parties
    f0, f1 = fused(prm, s0, s1, tensor_id=6)
    p0, p1, msgs = parties(prm, s0, s1, tensor_id=6)
    assert torch.equal(f0, p0) and torch.equal(f1, p1)
    assert msgs["w0"].numel() == (lx + 1) * padded_groups(n) * (lx + 1)
    assert ctx.parties_status() == 0
    es0, es1 = O.share(ring, masked(x, ring), SEED, 5)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1, aud = ofn(O.params(ring, lx, c), es0, es1, SEED, 6, audit=True, threads=8)
    assert np.array_equal(to_np(p0).astype(np.uint64), e0)
    assert np.array_equal(to_np(p1).astype(np.uint64), e1)
    assert np.array_equal(unpack_w(to_np(msgs["w0"]), lx, n), aud["w0"].astype(np.uint64))
    assert np.array_equal(unpack_w(to_np(msgs["w1"]), lx, n), aud["w1"].astype(np.uint64))
    assert np.array_equal(to_np(msgs["reply"]).astype(np.uint64), aud["reply"])
    if op == "relu":
        for k in ("open0", "open1", "pre_c1"):
            assert np.array_equal(to_np(msgs[k]).astype(np.uint64), aud[k])
    ctx.close()


def test_p2_wait_runs_out_and_reports():
    """P2's bounded wait for its bulk copies: with the test hook on, no copy
    is issued, the wait gives up after its limit, the call reports
    BC_ETIMEOUT through the status word, and the context stays usable."""
    ctx = Context(SEED)
    n = 700                      # three CTAs, the last one partial
    x = W.magnitude_bounded_ints(n, 20, seed=3)
    s0, s1 = ctx.share(64, torch.from_numpy(x).cuda(), 5)
    prm = Params(64, 24, 0)
    assert ctx.parties_status() == 0
    ctx.test_drop_p2_copies(True)
    ctx.relu_parties(prm, s0, s1, tensor_id=6)
    assert ctx.parties_status() == -4          # BC_ETIMEOUT
    assert ctx.parties_status() == 0           # reading clears it
    ctx.test_drop_p2_copies(False)
    p0, p1, _ = ctx.relu_parties(prm, s0, s1, tensor_id=6)
    f0, f1 = ctx.relu(prm, s0, s1, tensor_id=6)
    assert torch.equal(p0, f0) and torch.equal(p1, f1)
    assert ctx.parties_status() == 0
    ctx.close()


def test_unaligned_message_buffer_rejected():
    """The packed buffers are read by bulk copies: a buffer that is not
    16-byte aligned is rejected before anything is launched."""
    ctx = Context(SEED)
    n = 300
    x = W.magnitude_bounded_ints(n, 20, seed=4)
    s0, s1 = ctx.share(64, torch.from_numpy(x).cuda(), 5)
    prm = Params(64, 24, 0)
    msgs = ctx.party_buffers(prm, n)
    words = msgs["w0"].numel()
    base = torch.empty(words + 4, dtype=torch.int32, device=s0.device)
    msgs["w0"] = base[1:words + 1]             # 4 bytes past a 16-byte boundary
    with pytest.raises(BicoptorError):
        ctx.relu_parties(prm, s0, s1, tensor_id=6, msgs=msgs)
    ctx.close()


def test_parties_empty_input():
    ctx = Context(SEED)
    prm = Params(64, 24, 0)
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    assert ctx._lib.bc_party_msg_words(24, 0) == 0
    p0, p1, _ = ctx.relu_parties(prm, e, e, tensor_id=1)
    assert p0.numel() == 0 and p1.numel() == 0
    assert ctx.parties_status() == 0
    ctx.close()


# ---- P0, P1 and P2 as three processes (gloo through host memory, one GPU) ----

THREE_SEED = 0x3B0C_E550


def _three_worker(rank, port, out_dir, cases, transport="gloo"):
    import os as _os
    import torch.distributed as dist
    from paper_2309_04909_gb300 import Context, Params, workloads as W
    from paper_2309_04909_gb300.parties import (IpcTransport, PartyProcess, Transport,
                                                context_stages)
    _os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=3)
    torch.cuda.set_device(0)
    ctx = Context(THREE_SEED)
    ipc = IpcTransport(torch.device("cuda", 0)) if transport == "ipc" else None
    res = {}
    for ci, (ring, lx, c, mag, n, relu) in enumerate(cases):
        prm = Params(ring, lx, c)
        # the dealer's shares (every process derives the same ones; each party
        # keeps its own)
        x = W.magnitude_bounded_ints(n, mag, seed=ci)
        s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 50 + ci)
        share = (s0, s1, None)[rank]
        tr = ipc if ipc is not None else Transport(torch.device("cuda", 0), direct=False)
        tr.sent = {}
        ctx.reset_comm()
        pp = PartyProcess(rank, context_stages(ctx), tr)
        out = pp.run(prm, relu, share, n, 60 + ci)
        if transport == "ipc":            # the same call again through the same buffers
            torch.cuda.synchronize()
            first = None if out is None else out.clone()
            tr.sent = {}
            ctx.reset_comm()
            out = pp.run(prm, relu, share, n, 60 + ci)
            assert first is None or torch.equal(first, out)
        torch.cuda.synchronize()
        res[ci] = (None if out is None else out.cpu().numpy(), dict(tr.sent), ctx.comm())
    np.save(_os.path.join(out_dir, f"p{rank}.npy"), np.array([res], dtype=object),
            allow_pickle=True)
    del ipc
    torch.cuda.synchronize()
    dist.barrier()
    dist.destroy_process_group()
    ctx.close()


@pytest.mark.parametrize("transport", ["gloo", "ipc"])
def test_three_processes_match_fused_and_oracle(tmp_path, transport):
    """Each party in its own process and context: P0 and P1 send their
    packed w messages to P2 (and their openings to each other), P2 replies;
    every message moves through the transport into the receiver's memory:
    through host memory (gloo), or copied by the GPU into the receiver's own
    device buffer (CUDA IPC, twice through the same buffers).
    The output shares equal the fused kernel's and the oracle's bit for bit,
    and the three contexts' bit counters add up to the fused call's."""
    import socket
    import torch.multiprocessing as mp
    cases = [(64, 24, 0, 23, 10_007, True), (64, 24, 0, 23, 5_000, False),
             (32, 14, 4, 17, 3_001, True), (32, 9, 14, 22, 777, False), (64, 7, 0, 6, 1, True)]
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    mp.start_processes(_three_worker, args=(port, str(tmp_path), cases, transport), nprocs=3,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"p{k}.npy", allow_pickle=True)[0] for k in range(3)]
    ctx = Context(THREE_SEED)
    for ci, (ring, lx, c, mag, n, relu) in enumerate(cases):
        prm = Params(ring, lx, c)
        x = W.magnitude_bounded_ints(n, mag, seed=ci)
        s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 50 + ci)
        ctx.reset_comm()
        f0, f1 = (ctx.relu if relu else ctx.drelu)(prm, s0, s1, tensor_id=60 + ci)
        fused_comm = ctx.comm()
        assert np.array_equal(r[0][ci][0], f0.cpu().numpy()), ci
        assert np.array_equal(r[1][ci][0], f1.cpu().numpy()), ci
        es0, es1 = O.share(ring, masked(x, ring), THREE_SEED, 50 + ci)
        e0, e1 = (O.relu if relu else O.drelu)(O.params(ring, lx, c), es0, es1, THREE_SEED,
                                                60 + ci, threads=8)
        assert np.array_equal(r[0][ci][0].view(np.uint64 if ring > 32 else np.uint32)
                              .astype(np.uint64), e0)
        assert np.array_equal(r[1][ci][0].view(np.uint64 if ring > 32 else np.uint32)
                              .astype(np.uint64), e1)
        total = {k: sum(r[p][ci][2][k] for p in range(3)) for k in fused_comm}
        assert total == fused_comm, (ci, total, fused_comm)
        # bytes moved: the padded packed w buffers to P2, the ring lanes back
        wbytes = 4 * ctx._lib.bc_party_msg_words(lx, n)
        lane = 8 if ring > 32 else 4
        assert r[0][ci][1][(0, 2)] == wbytes and r[1][ci][1][(1, 2)] == wbytes
        assert r[2][ci][1][(2, 1)] == (2 if relu else 1) * n * lane
    ctx.close()
