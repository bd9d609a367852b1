"""Parity at the full sizes of the batched workloads, in the launch shapes the
benchmark times: the VGG-16 32x32 ReLU set of 128 images (1,664 tensors,
35,389,440 elements, l = 64) and the ResNet-18 224x224 set of 32 images in
both rings (1,088 tensors, 147,718,144 elements; l = 64 with (lx, c) = (24, 0)
and l = 32 with (14, 4)).  Sampled elements of many tensors are recomputed by
the oracle one by one; every element is checked against a property that
holds at any size (the reconstructed ReLU is x or 0, and max(x, 0) outside
the predicted exception set)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import Context, Params, workloads as W
from paper_2309_04909_gb300.batch import ReluBatch
from tests._util import cuda_ok, masked, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_0000_0005


def _check_sampled(ring, prm, allx, s0, s1, o0, o1, share_tid, spans, rng, tensors=40,
                   per=64):
    """spans: (tensor_id, offset, size) per tensor; checks `per` sampled
    elements of `tensors` sampled tensors against the oracle."""
    P = O.params(ring, prm.lx, prm.key_off)
    s0n, s1n, o0n, o1n = to_np(s0), to_np(s1), to_np(o0), to_np(o1)
    for k in rng.choice(len(spans), size=min(tensors, len(spans)), replace=False):
        tid, off, size = spans[k]
        j = np.sort(rng.choice(size, size=min(per, size), replace=False)).astype(np.uint64)
        g = j + np.uint64(off)
        es0, es1 = O.share(ring, masked(allx[g.astype(np.int64)], ring), SEED, share_tid, idx=g)
        assert np.array_equal(s0n[g.astype(np.int64)].astype(np.uint64), es0)
        assert np.array_equal(s1n[g.astype(np.int64)].astype(np.uint64), es1)
        e0, e1 = O.relu(P, es0, es1, SEED, tid, idx=j, threads=8)
        assert np.array_equal(o0n[g.astype(np.int64)].astype(np.uint64), e0), tid
        assert np.array_equal(o1n[g.astype(np.int64)].astype(np.uint64), e1), tid


def _check_property(ctx, ring, x_dev, o0, o1, min_exact):
    rec = ctx.reconstruct(ring, o0, o1).to(torch.int64)
    if ring < 64:          # sign-extend the l-bit values
        rec = torch.where(rec >= (1 << (ring - 1)), rec - (1 << ring), rec)
    assert bool(((rec == x_dev) | (rec == 0)).all())
    exact = (rec == torch.clamp(x_dev, min=0)).double().mean().item()
    assert exact >= min_exact, exact


@pytest.mark.parametrize("schedule", [1, 0])
def test_vgg16_batch128_full_size(schedule):
    ctx = Context(SEED)
    dev = torch.device("cuda")
    ts = W.vgg16_batch(128, seed=2)
    allx = np.concatenate([np.rint(np.ldexp(r, 16)).astype(np.int64) for r in ts.reals])
    assert allx.size == 35_389_440 and len(ts.sizes) == 1664
    xd = torch.from_numpy(allx).to(dev)
    s0, s1 = ctx.share(64, xd, tensor_id=11)
    o0, o1 = torch.empty_like(s0), torch.empty_like(s1)
    prm = Params(64, 24, 0)
    items, spans, off = [], [], 0
    for t, sz in enumerate(ts.sizes):
        items.append((prm, s0[off:off + sz], s1[off:off + sz], o0[off:off + sz],
                      o1[off:off + sz], 20000 + t))
        spans.append((20000 + t, off, sz))
        off += sz
    b = ReluBatch(ctx, items, schedule=schedule)
    b.run()
    torch.cuda.synchronize()
    assert ctx.batch_status() == 0
    _check_sampled(64, prm, allx, s0, s1, o0, o1, 11, spans, np.random.default_rng(schedule))
    _check_property(ctx, 64, xd, o0, o1, 0.9999)
    ctx.close()


def test_resnet18_batch32_mixed_rings_full_size():
    ctx = Context(SEED)
    dev = torch.device("cuda")
    ts = W.resnet18_mixed_batch(32, seed=3)
    assert ts.total == 147_718_144 and len(ts.sizes) == 1088
    items, parts = [], []
    for ring, frac, prm in ((64, 16, Params(64, 24, 0)), (32, 12, Params(32, 14, 4))):
        idx = [i for i in range(len(ts.sizes)) if ts.ring_bits[i] == ring]
        allx = np.concatenate([np.rint(np.ldexp(ts.reals[i], frac)).astype(np.int64)
                               for i in idx])
        xd = torch.from_numpy(allx).to(dev)
        s0, s1 = ctx.share(ring, xd, tensor_id=30 + ring)
        dt = torch.int64 if ring > 32 else torch.int32
        o0 = torch.empty(allx.size, dtype=dt, device=dev)
        o1 = torch.empty_like(o0)
        spans, off = [], 0
        for i in idx:
            sz = ts.sizes[i]
            items.append((prm, s0[off:off + sz], s1[off:off + sz], o0[off:off + sz],
                          o1[off:off + sz], 40000 + i))
            spans.append((40000 + i, off, sz))
            off += sz
        parts.append((ring, prm, allx, xd, s0, s1, o0, o1, spans))
    ts.reals = None
    b = ReluBatch(ctx, items, schedule=1)   # one launch per parameter group
    b.run()
    torch.cuda.synchronize()
    assert ctx.batch_status() == 0
    rng = np.random.default_rng(7)
    for ring, prm, allx, xd, s0, s1, o0, o1, spans in parts:
        _check_sampled(ring, prm, allx, s0, s1, o0, o1, 30 + ring, spans, rng)
        # l = 32, c = 4: |x| < 2^c may take either sign (reading 14), about 0.2 % here
        _check_property(ctx, ring, xd, o0, o1, 0.9999 if ring == 64 else 0.99)
    ctx.close()
