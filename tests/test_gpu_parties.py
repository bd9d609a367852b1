"""Party-separated DReLU/ReLU on the GPU: the three launches (P0/P1 local
work, P2, P0/P1 finish) exchange every message through device buffers and
give the fused kernel's outputs and the oracle's messages, bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import Context, Params, workloads as W
from tests._util import masked, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED = 0x9A27_1E5


def unpack_w(words: np.ndarray, lx: int, n: int) -> np.ndarray:
    """Inverse of the packed message layout: (n, lx+1) values."""
    B, L, G = lx + 1, lx + 1, (n + 31) // 32
    w = words.view(np.uint32).astype(np.uint64).reshape(L, G, B)
    bits = np.zeros((L, G, 32 * B), dtype=np.uint8)
    for b in range(32):
        bits[:, :, b::32] = ((w >> np.uint64(b)) & np.uint64(1)).astype(np.uint8)
    vals = np.zeros((L, G, 32), dtype=np.uint64)
    for b in range(B):
        vals |= bits[:, :, np.arange(32) * B + b].astype(np.uint64) << np.uint64(b)
    return vals.reshape(L, G * 32)[:, :n].T


CASES = [(64, 24, 0, 23, 10_007), (32, 9, 14, 22, 4_099), (32, 14, 4, 17, 3_000),
         (64, 7, 0, 6, 64), (64, 31, 2, 32, 1_001), (16, 5, 2, 6, 33)]


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
    assert msgs["w0"].numel() == (lx + 1) * ((n + 31) // 32) * (lx + 1)
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
