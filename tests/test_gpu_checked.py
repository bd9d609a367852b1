"""Checked mode: calls refuse share arrays whose lanes are not canonical
(bits at or above l set) and otherwise run unchanged; and the audit
comparison catches a single corrupted message."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import BicoptorError, Context, Params, workloads as W
from tests._util import cuda_ok, masked, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_0000_0004


@pytest.fixture()
def ctx():
    c = Context(SEED)
    yield c
    c.close()


def _shares(ctx, ring, n, tid, seed):
    x = W.magnitude_bounded_ints(n, ring - 6, seed=seed)
    return ctx.share(ring, torch.from_numpy(x).cuda(), tid)


@pytest.mark.parametrize("ring,lx,c", [(16, 5, 2), (48, 11, 2)])
def test_checked_refuses_noncanonical(ctx, ring, lx, c):
    n = 10_007
    s0, s1 = _shares(ctx, ring, n, 1, seed=ring)
    prm = Params(ring, lx, c)
    want = ctx.relu(prm, s0, s1, tensor_id=2)
    ctx.set_checked(True)
    got = ctx.relu(prm, s0, s1, tensor_id=2)          # canonical: runs, same result
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
    bad = s1.clone()
    bad[n - 3] |= 1 << ring                          # one lane with bit l set
    out = (torch.full_like(s0, 7), torch.full_like(s1, 7))
    with pytest.raises(BicoptorError):
        ctx.relu(prm, s0, bad, tensor_id=2, out=out)
    assert bool((out[0] == 7).all()) and bool((out[1] == 7).all())   # nothing launched
    with pytest.raises(BicoptorError):
        ctx.trunc_prob(ring, 3, bad, s0)
    with pytest.raises(BicoptorError):
        ctx.relu_batch_plan([(prm, s0, bad, out[0], out[1], 3)])
    ctx.set_checked(False)
    ctx.relu(prm, s0, bad, tensor_id=2, out=out)     # unchecked: runs (result unspecified)
    assert not bool((out[0] == 7).all())


def test_checked_full_rings_always_pass(ctx):
    """l = 32 and l = 64 lanes have no bits above l: checked calls run."""
    ctx.set_checked(True)
    for ring, lx, c in ((64, 24, 0), (32, 14, 4)):
        s0, s1 = _shares(ctx, ring, 4099, 5, seed=ring)
        ctx.relu(Params(ring, lx, c), s0, s1, tensor_id=6)


def test_audit_comparison_catches_one_corrupted_message(ctx):
    n, ring, lx = 3001, 64, 24
    x = W.magnitude_bounded_ints(n, 23, seed=9)
    s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 7)
    _, _, aud = ctx.drelu(Params(ring, lx, 0), s0, s1, tensor_id=8, audit=True)
    es0, es1 = O.share(ring, masked(x, ring), SEED, 7)
    _, _, eaud = O.drelu(O.params(ring, lx, 0), es0, es1, SEED, 8, audit=True, threads=8)
    w0 = to_np(aud["w0"]).reshape(n, lx + 1).copy()
    assert np.array_equal(w0, eaud["w0"])
    w0[1234, 7] ^= 1                                  # one bit of one message
    assert not np.array_equal(w0, eaud["w0"])
    assert np.argwhere(w0 != eaud["w0"]).tolist() == [[1234, 7]]


def test_checked_host_buffers(ctx):
    """The host-buffer step in checked mode refuses a non-canonical host lane
    before anything runs; canonical inputs give the unchecked result."""
    ring, k, n = 48, 8, 5001
    prm = Params(ring, 11, 2)
    x0, x1 = _shares(ctx, ring, n, 11, seed=1)
    y0, y1 = _shares(ctx, ring, n, 12, seed=2)
    hx = [t.cpu().pin_memory() for t in (x0, x1, y0, y1)]
    want = {nm: torch.empty(n, dtype=torch.int64).pin_memory() for nm in ("relu0", "relu1")}
    ctx.linear_relu_host(ring, k, prm, *hx, tensor_id=13, out=want)
    ctx.set_checked(True)
    got = {nm: torch.full((n,), 7, dtype=torch.int64).pin_memory() for nm in ("relu0", "relu1")}
    ctx.linear_relu_host(ring, k, prm, *hx, tensor_id=13, out=got)
    assert all(torch.equal(got[nm], want[nm]) for nm in got)
    bad = [t.clone().pin_memory() for t in hx]
    bad[2][77] |= 1 << ring
    fresh = {nm: torch.full((n,), 7, dtype=torch.int64).pin_memory() for nm in ("relu0", "relu1")}
    with pytest.raises(BicoptorError):
        ctx.linear_relu_host(ring, k, prm, *bad, tensor_id=13, out=fresh)
    assert all(bool((t == 7).all()) for t in fresh.values())
