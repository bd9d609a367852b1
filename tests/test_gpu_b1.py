"""The Bicoptor 1.0-style DReLU / ReLU on the GPU (the baseline Bicoptor 2.0
improves on): output shares and every message equal the oracle's bit for bit,
including a brute force over every x, every R and both flip bits at l = 8 and
l = 10, and the bits counted per party are (lx + 1) l."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import Context, Params, workloads as W
from tests._util import cuda_ok, masked, to_dev, to_np
from tests.test_gpu_edge_cases import _both_t_layout, _mask, _pairs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_00B1_0001
T = 8


@pytest.fixture(scope="module")
def ctx():
    c = Context(SEED)
    yield c
    c.close()


def _cmp(g, w):
    return np.array_equal(to_np(g).astype(np.uint64), w)


CASES = [(64, 24, 0, 23, 20_011), (64, 7, 24, 30, 10_007), (32, 14, 4, 17, 9_999),
         (32, 9, 14, 22, 4_096), (16, 5, 2, 6, 777), (8, 3, 1, 3, 300), (64, 31, 2, 32, 1_001),
         (64, 24, 0, 23, 1)]


@pytest.mark.parametrize("relu", [False, True])
@pytest.mark.parametrize("ring,lx,c,mag,n", CASES)
def test_b1_parity_with_messages(ctx, relu, ring, lx, c, mag, n):
    x = W.magnitude_bounded_ints(n, mag, seed=ring + lx + n)
    s0, s1 = ctx.share(ring, torch.from_numpy(x).cuda(), 11)
    prm = Params(ring, lx, c)
    fn = ctx.relu_b1 if relu else ctx.drelu_b1
    g0, g1, m0, m1 = fn(prm, s0, s1, tensor_id=12, messages=True)
    h0, h1 = fn(prm, s0, s1, tensor_id=12)                 # without the message buffers
    es0, es1 = O.share(ring, masked(x, ring), SEED, 11)
    e0, e1, w0, w1, dp = O.b1(O.params(ring, lx, c), es0, es1, SEED, 12, relu=relu, msgs=True,
                              threads=T)
    assert _cmp(g0, e0) and _cmp(g1, e1)
    assert torch.equal(g0, h0) and torch.equal(g1, h1)
    L = lx + 1
    assert np.array_equal(to_np(m0).astype(np.uint64).reshape(n, L), w0)
    assert np.array_equal(to_np(m1).astype(np.uint64).reshape(n, L), w1)


@pytest.mark.parametrize("ell,lx,c", [(8, 2, 0), (8, 3, 0), (8, 4, 0), (8, 3, 1), (8, 2, 2),
                                      (10, 5, 0), (10, 4, 2)])
def test_b1_bruteforce_every_x_every_r_both_t(ctx, ell, lx, c):
    full = np.arange(1 << ell, dtype=np.uint64)
    X, p0, p1 = _pairs(ell, full, full)
    tid = 3000 + ell * 100 + lx * 10 + c
    a0, a1, ia, ib, t = _both_t_layout(ell, p0, p1, tid, seed=tid)
    assert (t[ia] == 0).all() and (t[ib] == 1).all()
    prm, P = Params(ell, lx, c), O.params(ell, lx, c)
    s0, s1 = to_dev(a0, ell), to_dev(a1, ell)
    for relu in (False, True):
        fn = ctx.relu_b1 if relu else ctx.drelu_b1
        g0, g1 = fn(prm, s0, s1, tensor_id=tid)
        e0, e1 = O.b1(P, a0, a1, SEED, tid, relu=relu, threads=T)
        assert _cmp(g0, e0) and _cmp(g1, e1), relu


def test_b1_boundary_inputs(ctx):
    """Ring extremes and the key-window edges at l = 64, lx = 24, with R in
    {0, 1, 2^64 - 1, 2^63} and random R, under both flip bits."""
    ell, lx, c = 64, 24, 0
    xs = [0, 1, -1, (1 << 24) - 1, -((1 << 24) - 1), 1 << 24, -(1 << 24), 11_184_810,
          -11_184_810, 1 << 47, -(1 << 47), -(1 << 63), (1 << 63) - 1]
    rng = np.random.default_rng(64)
    rs = [0, 1, 2**64 - 1, 2**63] + [int(v) for v in rng.integers(0, 2**63, 12, dtype=np.uint64)]
    X, p0, p1 = _pairs(ell, [v & (2**64 - 1) for v in xs], rs)
    a0, a1, ia, ib, _ = _both_t_layout(ell, p0, p1, 77, min_n=50_000, seed=77)
    s0, s1 = to_dev(a0, ell), to_dev(a1, ell)
    P = O.params(ell, lx, c)
    for relu in (False, True):
        fn = ctx.relu_b1 if relu else ctx.drelu_b1
        g0, g1, m0, m1 = fn(Params(ell, lx, c), s0, s1, tensor_id=78, messages=True)
        e0, e1, w0, w1, _ = O.b1(P, a0, a1, SEED, 78, relu=relu, msgs=True, threads=T)
        assert _cmp(g0, e0) and _cmp(g1, e1)
        assert np.array_equal(to_np(m0).reshape(-1, lx + 1), w0)
    # with random R the sign inside the window is exact (a SecureML failure
    # has probability |x| / 2^64 per truncation); the extreme R values are
    # where it fails by construction (R = 2^64 - 1 wraps every positive x)
    d0, d1 = ctx.drelu_b1(Params(ell, lx, c), s0, s1, tensor_id=79)
    rec = (to_np(d0) + to_np(d1)) & _mask(64)
    xsig = X.view(np.int64)
    random_r = (np.arange(X.size) % len(rs)) >= 4
    ok = (xsig != 0) & (xsig > -(1 << 24)) & (xsig < (1 << 24)) & random_r   # no abs(-2^63)
    for pos in (ia, ib):
        assert (rec[pos][ok] == (xsig[ok] > 0)).all()


def test_b1_comm_counts_ring_elements(ctx):
    n = 1000
    x = W.magnitude_bounded_ints(n, 20, seed=5)
    s0, s1 = ctx.share(64, torch.from_numpy(x).cuda(), 1)
    for lx, c in ((24, 0), (7, 24)):
        ctx.reset_comm()
        ctx.drelu_b1(Params(64, lx, c), s0, s1, tensor_id=2)
        cm = ctx.comm()
        assert cm["p0_to_p2"] == n * (lx + 1) * 64 and cm["p1_to_p2"] == n * (lx + 1) * 64
        ctx.reset_comm()
        ctx.drelu(Params(64, lx, c), s0, s1, tensor_id=2)
        assert ctx.comm()["p0_to_p2"] == n * (lx + 1) * (lx + 1)   # Bicoptor 2.0


def test_b1_invalid_parameters(ctx):
    from paper_2309_04909_gb300 import BicoptorError
    s = torch.zeros(16, dtype=torch.int64, device="cuda")
    for prm in (Params(64, 32, 0), Params(64, 24, 40), Params(65, 8, 0), Params(64, 0, 0)):
        with pytest.raises(BicoptorError):
            ctx.drelu_b1(prm, s, s, tensor_id=1)
