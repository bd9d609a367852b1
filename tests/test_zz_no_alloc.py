"""bc_relu_batch_static: the batched ReLU for callers that may not allocate
device memory (e.g. a plugin inside a serving engine that owns all device
memory, or a loop under a fixed memory budget).  Called through the C-ABI, it
must give exactly the results of the context-based batched entry point,
call after call, although its scratch lives in one fixed device array that
every call reuses; it must leave the device's free memory unchanged, report
its status word, and refuse a capturing stream.  Collected last so a failure
here comes after every other test has run."""
import numpy as np
import pytest
import torch

from paper_2309_04909_gb300 import (BicoptorError, Context, Params, relu_batch_static,
                                    relu_batch_static_status)
from paper_2309_04909_gb300 import workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SEED = 0x0A11_0C00_5EED


def _batch(ctx, specs, seed):
    rng = np.random.default_rng(seed)
    items = []
    for ti, (ring, lx, c, mag) in enumerate(specs):
        n = int(rng.integers(1, 60_000))
        x = W.magnitude_bounded_ints(n, mag, seed=seed * 100 + ti)
        s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 40 + ti)
        dt = torch.int64 if ring > 32 else torch.int32
        o0 = torch.zeros(n, dtype=dt, device="cuda")
        o1 = torch.zeros(n, dtype=dt, device="cuda")
        items.append((Params(ring, lx, c), s0, s1, o0, o1, 7000 + ti, ti % 2))
    return items


def _reference(ctx, items):
    ref = [(torch.empty_like(it[3]), torch.empty_like(it[4])) for it in items]
    plan = [(it[0], it[1], it[2], r[0], r[1], it[5], it[6]) for it, r in zip(items, ref)]
    ctx.relu_batch_plan(plan, tile_elems=2048)
    ctx.relu_batch_run()
    torch.cuda.synchronize()
    return ref


def test_static_batch_matches_context_batch_twice():
    ctx = Context(SEED)
    specs_a = [(64, 24, 0, 23), (32, 14, 4, 17), (32, 9, 14, 22), (64, 7, 0, 6), (16, 5, 2, 6)]
    specs_b = [(64, 24, 0, 20), (64, 24, 0, 23), (32, 9, 14, 21)]
    for specs, seed, tile in ((specs_a, 1, 2048), (specs_b, 2, 0)):
        items = _batch(ctx, specs, seed)
        ref = _reference(ctx, items)
        relu_batch_static(SEED, items, tile_elems=tile)
        assert relu_batch_static_status() == 0
        for it, (r0, r1) in zip(items, ref):
            assert torch.equal(it[3], r0) and torch.equal(it[4], r1)
    ctx.close()


def test_static_batch_rejects_oversized_requests():
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    items = [(Params(64, 24, 0), x, x, x, x, i) for i in range(257)]
    with pytest.raises(BicoptorError, match="capacity"):
        relu_batch_static(SEED, items)
    big = torch.zeros(16385 * 16 + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(BicoptorError, match="capacity"):
        relu_batch_static(SEED, [(Params(64, 24, 0), big, big, big, big, 1)], tile_elems=16)


def test_static_batch_allocates_nothing_drelu_only():
    """After a first call, further calls (ReLU and DReLU-only batches) leave
    the device's free memory exactly unchanged, and match the context path."""
    ctx = Context(SEED)
    specs = [(64, 24, 0, 23), (32, 9, 14, 22), (64, 7, 0, 6)]
    relu_items = _batch(ctx, specs, 3)
    drelu_items = [it[:6] + (1,) for it in _batch(ctx, specs, 4)]
    refs = [_reference(ctx, its) for its in (relu_items, drelu_items)]
    relu_batch_static(SEED, relu_items)            # first call on the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for its, ref in zip((relu_items, drelu_items), refs):
            for it in its:
                it[3].zero_()
                it[4].zero_()
            relu_batch_static(SEED, its)
            assert relu_batch_static_status() == 0
            for it, (r0, r1) in zip(its, ref):
                assert torch.equal(it[3], r0) and torch.equal(it[4], r1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()


def test_static_batch_rejects_more_than_32_parameter_groups():
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    o = [torch.zeros(4, dtype=torch.int64, device="cuda") for _ in range(68)]
    items = [(Params(64, lx, 0), x, x, o[2 * lx], o[2 * lx + 1], lx) for lx in range(1, 32)]
    items += [(Params(63, lx, 0), x, x, o[62 + 2 * lx], o[63 + 2 * lx], 100 + lx)
              for lx in (1, 2)]
    with pytest.raises(BicoptorError, match="capacity"):
        relu_batch_static(SEED, items)
    relu_batch_static(SEED, items[:32])             # 32 groups fit
    assert relu_batch_static_status() == 0


def test_static_batch_refuses_a_capturing_stream():
    """Its tables come from host staging that the next call overwrites, so a
    call on a stream under capture is refused and leaves the outputs alone."""
    import ctypes
    from paper_2309_04909_gb300 import _native
    from paper_2309_04909_gb300._native import TensorDesc
    ctx = Context(SEED)
    items = _batch(ctx, [(64, 24, 0, 23)], 5)
    lib = _native.lib()
    arr = (TensorDesc * 1)()
    prm, s0, s1, o0, o1, tid, op = items[0]
    arr[0] = TensorDesc(s0.data_ptr(), s1.data_ptr(), o0.data_ptr(), o1.data_ptr(), s0.numel(),
                        tid, op, prm.c_struct(), 0)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        rc = lib.bc_relu_batch_static(SEED, 0, ctypes.c_void_p(side.cuda_stream), arr, 1, 0)
        rs = lib.bc_relu_batch_static_status(0, ctypes.c_void_p(side.cuda_stream))
        marker.add_(1)                              # the graph's only node
    assert rc == -1 and rs == -1
    g.replay()
    torch.cuda.synchronize()
    assert marker.item() == 1
    assert not bool(o0.any()) and not bool(o1.any())
    relu_batch_static(SEED, items)                  # the same call outside capture runs
    assert relu_batch_static_status() == 0 and bool(o0.any())
    ctx.close()
