"""bc_relu_batch_static: the batched ReLU for callers that may not allocate
device memory (e.g. a plugin inside a serving engine that owns all device
memory, or a loop under a fixed memory budget).  Called through the C-ABI, it
must give exactly the results of the context-based batched entry point,
call after call, although its scratch lives in one fixed device array that
every call reuses.  Collected last so a failure here comes after every other
test has run."""
import numpy as np
import pytest
import torch

from paper_2309_04909_gb300 import BicoptorError, Context, Params, relu_batch_static
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
        torch.cuda.synchronize()
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
