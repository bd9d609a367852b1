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
