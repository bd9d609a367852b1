"""Parity of the fused step (Beaver product -> Alg. smltrc / Alg. newtrc ->
Alg. relu in one kernel) with the oracle's chain of the four operations, on
device buffers and through both host-buffer paths.

Integer protocol: every comparison is bit-exact.  Sizes span many CTAs and end
on a ragged tail.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import BicoptorError, Context, Params, workloads as W
from tests._util import cuda_ok, masked, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_0000_0003
NAMES = ("prod0", "prod1", "trc0", "trc1", "det0", "det1", "relu0", "relu1")


@pytest.fixture(scope="module")
def ctx():
    c = Context(SEED)
    yield c
    c.close()


def _case(ctx, ring, k, lx, c, n, mag, tid):
    """Shares of two seeded inputs, the fused outputs, and the oracle chain."""
    x = W.magnitude_bounded_ints(n, mag, seed=tid)
    y = W.magnitude_bounded_ints(n, mag, seed=tid + 1)
    s = [ctx.share(ring, torch.from_numpy(v).cuda(), t) for v, t in ((x, tid), (y, tid + 1))]
    ex0, ex1 = O.share(ring, masked(x, ring), SEED, tid)
    ey0, ey1 = O.share(ring, masked(y, ring), SEED, tid + 1)
    p0, p1 = O.mul_beaver(ring, ex0, ex1, ey0, ey1, SEED, tid + 2)
    t0, t1 = O.trunc_prob(ring, k, p0, p1)
    d0, d1 = O.trunc_det(ring, k, 0, p0, p1)
    r0, r1 = O.relu(O.params(ring, lx, c), t0, t1, SEED, tid + 3, threads=8)
    want = dict(zip(NAMES, (p0, p1, t0, t1, d0, d1, r0, r1)))
    return s[0], s[1], want


# (ring, k, lx, c, magnitude bits): the benchmark's configuration, a 32-bit
# ring, deterministic-truncation lanes narrower than the ring (l - k <= 32 on
# 64-bit lanes), and a key width with no specialised kernel
CASES = [(64, 16, 24, 0, 20), (32, 12, 14, 4, 10), (64, 40, 7, 0, 24), (64, 16, 20, 3, 20),
         (48, 8, 11, 2, 14)]


@pytest.mark.parametrize("ring,k,lx,c,mag", CASES)
def test_fused_step_matches_oracle_chain(ctx, ring, k, lx, c, mag):
    n = 70_001
    (x0, x1), (y0, y1), want = _case(ctx, ring, k, lx, c, n, mag, tid=100 + ring + k)
    prm = Params(ring, lx, c)
    got = ctx.linear_relu(ring, k, prm, x0, x1, y0, y1, tensor_id=102 + ring + k)
    for nm in NAMES:
        assert np.array_equal(to_np(got[nm]).astype(np.uint64), want[nm]), nm


def test_fused_step_optional_outputs(ctx):
    """Only the ReLU written; then ReLU and det.  Results equal the full call."""
    ring, k, n = 64, 16, 33_333
    (x0, x1), (y0, y1), want = _case(ctx, ring, k, 24, 0, n, 20, tid=300)
    prm = Params(ring, 24, 0)
    only = ctx.linear_relu_buffers(ring, k, n, names=("relu0", "relu1"))
    ctx.linear_relu(ring, k, prm, x0, x1, y0, y1, tensor_id=302, work=only)
    for nm in ("relu0", "relu1"):
        assert np.array_equal(to_np(only[nm]).astype(np.uint64), want[nm]), nm
    some = ctx.linear_relu_buffers(ring, k, n, names=("det0", "det1", "relu0", "relu1"))
    ctx.linear_relu(ring, k, prm, x0, x1, y0, y1, tensor_id=302, work=some)
    for nm in some:
        assert np.array_equal(to_np(some[nm]).astype(np.uint64), want[nm]), nm
    # one of a pair missing is an argument error, nothing launched
    bad = ctx.linear_relu_buffers(ring, k, n, names=("det0", "relu0", "relu1"))
    with pytest.raises(BicoptorError):
        ctx.linear_relu(ring, k, prm, x0, x1, y0, y1, tensor_id=302, work=bad)


def test_fused_step_empty(ctx):
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    got = ctx.linear_relu(64, 16, Params(64, 24, 0), e, e, e, e, tensor_id=1)
    assert all(t.numel() == 0 for t in got.values())


@pytest.mark.parametrize("path", ["auto", "direct", "staged", "pageable"])
def test_host_paths(ctx, path):
    """Host buffers in and out: the direct path (kernel loads and stores
    pinned memory), the staged path (chunked copies on four streams, chunk
    not dividing n so element offsets matter), and pageable buffers (AUTO
    falls back to staging)."""
    ring, k, n = 64, 16, 50_021
    (x0, x1), (y0, y1), want = _case(ctx, ring, k, 24, 0, n, 20, tid=400)
    prm = Params(ring, 24, 0)
    pin = path != "pageable"
    hx = [t.cpu().pin_memory() if pin else t.cpu() for t in (x0, x1, y0, y1)]
    out = {nm: torch.empty(n, dtype=torch.int64) for nm in ("relu0", "relu1", "det0", "det1")}
    if pin:
        out = {nm: t.pin_memory() for nm, t in out.items()}
    ctx.reserve(12_000)
    mode = {"auto": ctx.HOST_AUTO, "direct": ctx.HOST_DIRECT, "staged": ctx.HOST_STAGED,
            "pageable": ctx.HOST_AUTO}[path]
    ctx.set_host_path(mode)
    try:
        ctx.linear_relu_host(ring, k, prm, *hx, tensor_id=402, out=out)
    finally:
        ctx.set_host_path(ctx.HOST_AUTO)
    for nm, t in out.items():
        assert np.array_equal(t.numpy().view(np.uint64), want[nm]), nm


def test_host_direct_rejects_pageable(ctx):
    """HOST_DIRECT with a buffer that is not mapped page-locked memory is an
    argument error, found on the host before any launch."""
    n = 1000
    hx = [torch.zeros(n, dtype=torch.int64) for _ in range(4)]
    out = {nm: torch.empty(n, dtype=torch.int64) for nm in ("relu0", "relu1")}
    ctx.set_host_path(ctx.HOST_DIRECT)
    try:
        with pytest.raises(BicoptorError):
            ctx.linear_relu_host(64, 16, Params(64, 24, 0), *hx, tensor_id=1, out=out)
    finally:
        ctx.set_host_path(ctx.HOST_AUTO)


def test_host_path_value_checked(ctx):
    for bad in (-1, 3, 99):
        with pytest.raises(BicoptorError):
            ctx.set_host_path(bad)
    ctx.set_host_path(ctx.HOST_AUTO)
