"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Integer protocol: every comparison is bit-exact.  Sizes span many CTAs and
end on a ragged tail.  The full-size workloads are compared element by element
in test_gpu_configs.py, the exhaustive and boundary inputs in
test_gpu_edge_cases.py.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2309_04909_gb300 import Context, Params, workloads as W
from tests._util import cuda_ok, encode_np, masked, to_dev, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_0000_0001


@pytest.fixture(scope="module")
def ctx():
    c = Context(SEED)
    yield c
    c.close()


def _shares(ctx, bits, x_int, tid):
    xg = torch.from_numpy(x_int.astype(np.int64)).cuda()
    s0, s1 = ctx.share(bits, xg, tid)
    return s0, s1


@pytest.mark.parametrize("bits", [8, 16, 31, 32, 33, 48, 64])
@pytest.mark.parametrize("n", [0, 1, 5, 10007, 155_651])
def test_share_reconstruct(ctx, bits, n):
    x = W.magnitude_bounded_ints(n, min(bits - 2, 40), seed=bits * 7 + n)
    s0, s1 = _shares(ctx, bits, x, tid=3)
    e0, e1 = O.share(bits, masked(x, bits), seed=SEED, tid=3)
    assert np.array_equal(to_np(s0), e0.astype(to_np(s0).dtype))
    assert np.array_equal(to_np(s1), e1.astype(to_np(s1).dtype))
    rec = ctx.reconstruct(bits, s0, s1)
    assert np.array_equal(to_np(rec).astype(np.uint64), masked(x, bits))


@pytest.mark.parametrize("bits,k", [(64, 16), (64, 1), (64, 63), (32, 12), (16, 4), (8, 4), (40, 7)])
def test_trunc_prob(ctx, bits, k):
    n = 100_003
    rng = np.random.default_rng(bits + k)
    a = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=n, dtype=np.uint64)
    b = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(3)
    a, b = masked(a, bits), masked(b, bits)
    o0, o1 = ctx.trunc_prob(bits, k, to_dev(a, bits), to_dev(b, bits))
    e0, e1 = O.trunc_prob(bits, k, a, b)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


@pytest.mark.parametrize("bits,k1,k2", [(64, 16, 0), (64, 16, 16), (64, 3, 40), (64, 0, 8),
                                        (32, 4, 3), (32, 12, 0), (8, 4, 1), (48, 10, 10)])
def test_trunc_det(ctx, bits, k1, k2):
    n = 77_777
    rng = np.random.default_rng(bits * 3 + k1 + k2)
    a = masked(rng.integers(0, 2**64, size=n, dtype=np.uint64), bits)
    b = masked(rng.integers(0, 2**64, size=n, dtype=np.uint64), bits)
    o0, o1 = ctx.trunc_det(bits, k1, k2, to_dev(a, bits), to_dev(b, bits))
    e0, e1 = O.trunc_det(bits, k1, k2, a, b)
    assert to_np(o0).dtype == (np.uint64 if bits - k1 - k2 > 32 else np.uint32)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


@pytest.mark.parametrize("lp", [1, 5, 9, 14, 24, 31])
def test_mod_switch(ctx, lp):
    n = 50_001
    rng = np.random.default_rng(lp)
    a = masked(rng.integers(0, 2**32, size=n, dtype=np.uint64), lp)
    b = masked(rng.integers(0, 2**32, size=n, dtype=np.uint64), lp)
    b[:100] = (np.uint64(1 << lp) - a[:100]) & np.uint64((1 << lp) - 1)   # zeros
    for p in (O.prime_above(lp),):
        o0, o1 = ctx.mod_switch(lp, p, to_dev(a, 32), to_dev(b, 32))
        e0, e1 = O.mod_switch(lp, p, a, b)
        assert np.array_equal(to_np(o0), e0)
        assert np.array_equal(to_np(o1), e1)


@pytest.mark.parametrize("bits", [64, 32, 16])
def test_mul_beaver(ctx, bits):
    n = 65_537
    x = W.magnitude_bounded_ints(n, bits // 2 - 2, seed=1)
    y = W.magnitude_bounded_ints(n, bits // 2 - 2, seed=2)
    x0, x1 = _shares(ctx, bits, x, 10)
    y0, y1 = _shares(ctx, bits, y, 11)
    o0, o1 = ctx.mul_beaver(bits, x0, x1, y0, y1, tensor_id=12)
    ex0, ex1 = O.share(bits, masked(x, bits), SEED, 10)
    ey0, ey1 = O.share(bits, masked(y, bits), SEED, 11)
    e0, e1 = O.mul_beaver(bits, ex0, ex1, ey0, ey1, SEED, 12)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


PROTO = [
    # (ring, lx, c, magnitude bits of inputs, n)
    (64, 24, 0, 23, 40_013),
    (32, 9, 14, 22, 65_536),
    (32, 14, 4, 17, 30_011),
    (64, 7, 0, 6, 9_999),       # the paper's lx = 7 (5+2)
    (64, 31, 2, 32, 5_003),     # widest window: p > 2^31
    (16, 5, 2, 6, 7_001),       # generic-lx kernel
    (8, 3, 0, 2, 4_097),
    (33, 10, 3, 12, 3_001),
    (2, 1, 0, 1, 1_001),        # smallest ring: l = 2, one key bit, p = 3
    (4, 1, 1, 2, 999),          # one key bit above the offset
]


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", PROTO)
def test_protocol_parity_with_audit(ctx, op, ring, lx, c, mag, n):
    x = W.magnitude_bounded_ints(n, mag, seed=ring + lx + c)
    tid = 100 + lx
    s0, s1 = _shares(ctx, ring, x, tid)
    prm = Params(ring, lx, c)
    P = O.params(ring, lx, c)
    fn = ctx.drelu if op == "drelu" else ctx.relu
    o0, o1, aud = fn(prm, s0, s1, tensor_id=tid + 1, audit=True)
    es0, es1 = O.share(ring, masked(x, ring), SEED, tid)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1, eaud = ofn(P, es0, es1, SEED, tid + 1, audit=True, threads=8)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)
    L = lx + 1
    assert np.array_equal(to_np(aud["w0"]).reshape(n, L), eaud["w0"])
    assert np.array_equal(to_np(aud["w1"]).reshape(n, L), eaud["w1"])
    assert np.array_equal(to_np(aud["t"]), eaud["t"])
    assert np.array_equal(to_np(aud["dprime"]), eaud["dprime"])
    assert np.array_equal(to_np(aud["reply"]).astype(np.uint64), eaud["reply"])
    if op == "relu":
        for k in ("open0", "open1", "pre_c1"):
            assert np.array_equal(to_np(aud[k]).astype(np.uint64), eaud[k])


# The kernels compiled for fixed key widths (lx = 24 and 7 at l = 64, 14 and 9
# at l = 32) at key offsets the configurations above do not reach: at l = 64
# on both sides of c + lx = 32 (below it the window is one funnel shift of the
# lane's two words), and l = 32 at c = 0.  The flipped shares are shifted by c
# once per element, so every window of step 3 depends on it.
OFFSETS = [(64, 24, 5, 28, 20_011), (64, 24, 9, 32, 20_011), (64, 7, 24, 30, 9_999),
           (64, 7, 30, 36, 9_999), (32, 14, 0, 13, 9_999), (32, 9, 0, 8, 9_999)]


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", OFFSETS)
def test_fixed_width_kernels_at_key_offsets(ctx, op, ring, lx, c, mag, n):
    """Single-tensor kernel with and without the audit, and the batched grid
    kernel, against the oracle element by element (messages too)."""
    x = W.magnitude_bounded_ints(n, mag, seed=ring * 5 + lx * 3 + c)
    tid = 300 + lx + c
    s0, s1 = _shares(ctx, ring, x, tid)
    prm, P = Params(ring, lx, c), O.params(ring, lx, c)
    es0, es1 = O.share(ring, masked(x, ring), SEED, tid)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1, eaud = ofn(P, es0, es1, SEED, tid + 1, audit=True, threads=8)
    fn = ctx.drelu if op == "drelu" else ctx.relu
    o0, o1, aud = fn(prm, s0, s1, tensor_id=tid + 1, audit=True)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)
    L = lx + 1
    assert np.array_equal(to_np(aud["w0"]).reshape(n, L), eaud["w0"])
    assert np.array_equal(to_np(aud["w1"]).reshape(n, L), eaud["w1"])
    assert np.array_equal(to_np(aud["dprime"]), eaud["dprime"])
    o0, o1 = fn(prm, s0, s1, tensor_id=tid + 1)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)
    b0, b1 = torch.empty_like(s0), torch.empty_like(s1)
    ctx.relu_batch_plan([(prm, s0, s1, b0, b1, tid + 1, 1 if op == "drelu" else 0)],
                        schedule=1)
    ctx.relu_batch_run()
    assert ctx.batch_status() == 0
    assert np.array_equal(to_np(b0).astype(np.uint64), e0)
    assert np.array_equal(to_np(b1).astype(np.uint64), e1)


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", PROTO[:4])
def test_protocol_parity_no_audit(ctx, op, ring, lx, c, mag, n):
    """The kernel without message materialisation gives the same outputs."""
    x = W.magnitude_bounded_ints(n, mag, seed=ring * 3 + lx)
    s0, s1 = _shares(ctx, ring, x, 7)
    fn = ctx.drelu if op == "drelu" else ctx.relu
    o0, o1 = fn(Params(ring, lx, c), s0, s1, tensor_id=8)
    es0, es1 = O.share(ring, masked(x, ring), SEED, 7)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1 = ofn(O.params(ring, lx, c), es0, es1, SEED, 8, threads=8)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


# The largest prime below 2^32, a valid p for lx = 31 (2^31 < p < 2^32).  The
# Montgomery quotient of the masking then needs 33 bits.
P_MAX32 = 4294967291


@pytest.mark.parametrize("op", ["drelu", "relu"])
def test_largest_prime_parity(ctx, op):
    """lx = 31 with a caller-chosen p near 2^32: outputs and every masked
    message equal the oracle's, in the fused kernel and the party-separated
    launches."""
    ring, lx, c, n = 64, 31, 2, 20_011
    x = W.magnitude_bounded_ints(n, 32, seed=77)
    s0, s1 = _shares(ctx, ring, x, 60)
    prm = Params(ring, lx, c, p=P_MAX32)
    P = O.params(ring, lx, c, p=P_MAX32)
    fn = ctx.drelu if op == "drelu" else ctx.relu
    o0, o1, aud = fn(prm, s0, s1, tensor_id=61, audit=True)
    es0, es1 = O.share(ring, masked(x, ring), SEED, 60)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1, eaud = ofn(P, es0, es1, SEED, 61, audit=True, threads=8)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)
    assert np.array_equal(to_np(aud["w0"]).reshape(n, lx + 1), eaud["w0"])
    assert np.array_equal(to_np(aud["w1"]).reshape(n, lx + 1), eaud["w1"])
    parties = ctx.drelu_parties if op == "drelu" else ctx.relu_parties
    p0, p1, _ = parties(prm, s0, s1, tensor_id=61)
    assert np.array_equal(to_np(p0).astype(np.uint64), e0)
    assert np.array_equal(to_np(p1).astype(np.uint64), e1)


def test_largest_prime_rss(ctx):
    ring, lx, c, n = 64, 31, 2, 9_001
    x = W.magnitude_bounded_ints(n, 32, seed=78)
    rng = np.random.default_rng(78)
    x0 = rng.integers(0, 2**63, n, dtype=np.uint64)
    x1 = rng.integers(0, 2**63, n, dtype=np.uint64)
    x2 = x.astype(np.uint64) - x0 - x1
    ys = ctx.rss_relu(Params(ring, lx, c, p=P_MAX32), to_dev(x0, ring), to_dev(x1, ring),
                      to_dev(x2, ring), tensor_id=62)
    e = O.rss_drelu(O.params(ring, lx, c, p=P_MAX32), x0, x1, x2, SEED, 62, relu=True,
                    threads=8)
    for g, w in zip(ys, e[:3]):
        assert np.array_equal(to_np(g).astype(np.uint64), w)


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", [(64, 24, 0, 23, 1), (64, 24, 0, 23, 63),
                                            (64, 24, 0, 23, 1000), (64, 7, 0, 6, 5001),
                                            (32, 14, 4, 17, 777), (16, 5, 2, 6, 300),
                                            (64, 20, 3, 22, 4097), (32, 9, 14, 22, 70_001)])
def test_small_batch_parity(ctx, op, ring, lx, c, mag, n):
    """Small launches (the four-lanes-per-element kernel, partial warps and
    CTAs included) are bit-identical to the oracle."""
    x = W.magnitude_bounded_ints(n, mag, seed=n + lx)
    s0, s1 = _shares(ctx, ring, x, 40)
    fn = ctx.drelu if op == "drelu" else ctx.relu
    o0, o1 = fn(Params(ring, lx, c), s0, s1, tensor_id=41)
    es0, es1 = O.share(ring, masked(x, ring), SEED, 40)
    ofn = O.drelu if op == "drelu" else O.relu
    e0, e1 = ofn(O.params(ring, lx, c), es0, es1, SEED, 41, threads=8)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


def test_protocol_empty_and_single(ctx):
    prm = Params(64, 24, 0)
    z = torch.empty(0, dtype=torch.int64, device="cuda")
    o0, o1 = ctx.relu(prm, z, z, tensor_id=1)
    assert o0.numel() == 0
    x = np.array([-5 * 2**16], dtype=np.int64)
    s0, s1 = _shares(ctx, 64, x, 4)
    o0, o1 = ctx.relu(prm, s0, s1, tensor_id=5)
    es0, es1 = O.share(64, masked(x, 64), SEED, 4)
    e0, e1 = O.relu(O.params(64, 24, 0), es0, es1, SEED, 5)
    assert to_np(o0)[0] == e0[0] and to_np(o1)[0] == e1[0]


def test_invalid_parameters_rejected(ctx):
    from paper_2309_04909_gb300 import BicoptorError
    s = torch.zeros(16, dtype=torch.int64, device="cuda")
    for prm in (Params(64, 32, 0), Params(64, 24, 17), Params(64, 24, 0, p=16777217),
                Params(64, 24, 0, p=2**24 - 3), Params(65, 8, 0), Params(64, 0, 0)):
        with pytest.raises(BicoptorError):
            ctx.relu(prm, s, s, tensor_id=1)
    with pytest.raises(BicoptorError):
        ctx.trunc_prob(64, 64, s, s)
    with pytest.raises(BicoptorError):
        ctx.mod_switch(9, 512, s.to(torch.int32), s.to(torch.int32))


def test_comm_counters(ctx):
    ctx.reset_comm()
    n = 1000
    x = W.magnitude_bounded_ints(n, 20, seed=5)
    s0, s1 = _shares(ctx, 64, x, 1)
    ctx.drelu(Params(64, 24, 0), s0, s1, tensor_id=2)
    c = ctx.comm()
    assert c["p0_to_p2"] == n * 25 * 25 and c["p1_to_p2"] == n * 25 * 25   # (lx+1)^2 bits
    assert c["p2_to_p1"] == n * 64 and c["p2_to_p0"] == 0 and c["rounds"] == 2
    ctx.reset_comm()
    ctx.relu(Params(64, 7, 0), s0, s1, tensor_id=2)
    c = ctx.comm()
    assert c["p0_to_p2"] == n * 64   # the paper's 8 * 8 = 64 bits at lx = 7
    assert c["p2_to_p0"] == n * 64 and c["p0_to_p1"] == n * 64 and c["pre_p2_to_p1"] == n * 64


def test_count_trunc_failures(ctx):
    n = 1 << 18
    x = W.magnitude_bounded_ints(n, 60, seed=9)
    s0, s1 = _shares(ctx, 64, x, 2)
    o0, o1 = ctx.trunc_prob(64, 16, s0, s1)
    xg = torch.from_numpy(x).cuda()
    got = ctx.count_trunc_failures(64, 16, xg, o0, o1)
    es0, es1 = O.share(64, masked(x, 64), SEED, 2)
    e0, e1 = O.trunc_prob(64, 16, es0, es1)
    rec = O.to_signed(O.reconstruct(64, e0, e1), 64)
    d = (rec.astype(object) - (x >> 16).astype(object)) % 2**64
    want = int(sum(1 for v in d if v not in (0, 1, 2**64 - 1)))
    assert got == want and got > 0
    d0, d1 = ctx.trunc_det(64, 16, 0, s0, s1)
    assert ctx.count_trunc_failures(48, 16, xg, d0, d1) == 0


def test_linear_relu_chain(ctx):
    """Product -> truncation -> ReLU chain at reduced size: product, both truncations and
    the ReLU of the prob-truncated product, device and host-buffer paths."""
    n, f, k = 50_021, 16, 16
    X = W.gaussian_reals(n, 4.0, seed=1, stream=0)
    Y = W.gaussian_reals(n, 4.0, seed=1, stream=1)
    xi, yi = encode_np(X, f), encode_np(Y, f)
    x0, x1 = _shares(ctx, 64, xi, 20)
    y0, y1 = _shares(ctx, 64, yi, 21)
    prm = Params(64, 24, 0)
    w = ctx.linear_relu(64, k, prm, x0, x1, y0, y1, tensor_id=30)
    # oracle chain
    ex0, ex1 = O.share(64, masked(xi, 64), SEED, 20)
    ey0, ey1 = O.share(64, masked(yi, 64), SEED, 21)
    p0, p1 = O.mul_beaver(64, ex0, ex1, ey0, ey1, SEED, 30)
    t0, t1 = O.trunc_prob(64, k, p0, p1)
    d0, d1 = O.trunc_det(64, k, 0, p0, p1)
    r0, r1 = O.relu(O.params(64, 24, 0), t0, t1, SEED, 31, threads=8)
    for name, want in (("prod0", p0), ("prod1", p1), ("trc0", t0), ("trc1", t1), ("det0", d0),
                       ("det1", d1), ("relu0", r0), ("relu1", r1)):
        assert np.array_equal(to_np(w[name]).astype(np.uint64), want), name
    # host-buffer entry point, chunked so the element offsets matter
    ctx.reserve(12_000)
    hx = [t.cpu().pin_memory() for t in (x0, x1, y0, y1)]
    out = {nm: torch.empty(n, dtype=torch.int64).pin_memory() for nm in ("relu0", "relu1", "det0",
                                                                           "det1")}
    ctx.linear_relu_host(64, k, prm, *hx, tensor_id=30, out=out)
    for name, want in (("relu0", r0), ("relu1", r1), ("det0", d0), ("det1", d1)):
        assert np.array_equal(out[name].numpy().view(np.uint64), want), name


def test_batch_matches_single_calls(ctx):
    """Many tensors of uneven size and mixed rings in one persistent launch
    give bit-identical results to one call per tensor."""
    specs = [(64, 24, 0, 23), (32, 14, 4, 17), (32, 9, 14, 22), (64, 7, 0, 6), (16, 5, 2, 6)]
    rng = np.random.default_rng(0)
    items, singles = [], []
    for ti in range(23):
        ring, lx, c, mag = specs[ti % len(specs)]
        n = int(rng.integers(1, 40_000)) if ti % 4 else int(rng.integers(100_000, 200_000))
        x = W.magnitude_bounded_ints(n, mag, seed=ti)
        s0, s1 = _shares(ctx, ring, x, 500 + ti)
        prm = Params(ring, lx, c)
        o0, o1 = ctx._empty(n, ring), ctx._empty(n, ring)
        op = ti % 3 == 0  # some DReLU
        items.append((prm, s0, s1, o0, o1, 900 + ti, 1 if op else 0))
        fn = ctx.drelu if op else ctx.relu
        singles.append(fn(prm, s0, s1, tensor_id=900 + ti))
    # (tile, schedule, CTAs per SM, elements per thread, key-bit unroll)
    for tile, sched, cps, ept, unroll in ((0, 0, 0, 0, 0), (1000, 0, 2, 0, 3), (4096, 0, 1, 0, 1),
                                          (0, 1, 0, 0, 0), (0, 1, 0, 2, 1), (0, 1, 0, 4, 3),
                                          (0, 1, 0, 4, 2), (0, 1, 0, 1, 2), (0, 1, 0, 2, 0),
                                          (512, 0, 0, 0, 2)):
        for it in items:
            it[3].fill_(0)
            it[4].fill_(0)
        ctx.relu_batch_plan(items, tile_elems=tile, ctas_per_sm=cps, schedule=sched,
                            elems_per_thread=ept, slot_unroll=unroll)
        ctx.relu_batch_run()
        assert ctx.batch_status() == 0
        for it, (r0, r1) in zip(items, singles):
            assert torch.equal(it[3], r0) and torch.equal(it[4], r1)


@pytest.mark.parametrize("op", ["relu", "drelu"])
@pytest.mark.parametrize("start", [2**32 - 300, 2**40 + 12_345, 2**48 - 1000])
def test_element_index_above_32_bits(ctx, op, start):
    """A slice of a tensor at a large element offset: the element index needs
    more than 32 bits (the counter's fourth word carries bits 32..47), up to
    the last index the counter holds, 2^48 - 1.  The outputs match the oracle
    run at the same element indices."""
    ring, lx, c, n = 64, 24, 0, 1000
    x = W.magnitude_bounded_ints(n, 23, seed=91)
    s0, s1 = _shares(ctx, ring, x, 71)
    o0, o1 = ctx._empty(n, ring), ctx._empty(n, ring)
    items = [(Params(ring, lx, c), s0, s1, o0, o1, 72, 0 if op == "relu" else 1, start)]
    ctx.relu_batch_plan(items)
    ctx.relu_batch_run()
    assert ctx.batch_status() == 0
    es0, es1 = O.share(ring, masked(x, ring), SEED, 71)
    ofn = O.relu if op == "relu" else O.drelu
    idx = np.arange(start, start + n, dtype=np.uint64)
    e0, e1 = ofn(O.params(ring, lx, c), es0, es1, SEED, 72, idx=idx, threads=8)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


def test_element_index_past_48_bits_rejected(ctx):
    from paper_2309_04909_gb300 import BicoptorError
    s = torch.zeros(1000, dtype=torch.int64, device="cuda")
    o = torch.empty_like(s)
    ok = [(Params(64, 24, 0), s, s, o, o, 1, 0, 2**48 - 1000)]
    ctx.relu_batch_plan(ok)                    # ends exactly at 2^48
    for off in (2**48 - 999, 2**48, 2**64 - 1):
        with pytest.raises(BicoptorError):
            ctx.relu_batch_plan([(Params(64, 24, 0), s, s, o, o, 1, 0, off)])


def test_batch_config_out_of_range_rejected(ctx):
    from paper_2309_04909_gb300 import BicoptorError
    s = torch.zeros(1000, dtype=torch.int64, device="cuda")
    o = torch.empty_like(s)
    items = [(Params(64, 24, 0), s, s, o, o, 1)]
    for kw in ({"schedule": 1, "elems_per_thread": 3}, {"schedule": 1, "elems_per_thread": 8},
               {"slot_unroll": 4}, {"slot_unroll": -1}):
        with pytest.raises(BicoptorError):
            ctx.relu_batch_plan(items, **kw)


@pytest.mark.parametrize("bits,k,fixed", [(64, 16, 0), (64, 26, 1 << 26), (32, 12, 0), (16, 4, 0)])
def test_trunc_aby3(ctx, bits, k, fixed):
    n = 60_013
    x = W.magnitude_bounded_ints(n, bits - 3, seed=bits + k)
    s0, s1 = _shares(ctx, bits, x, 70)
    o0, o1 = ctx.trunc_aby3(bits, k, s0, s1, tensor_id=71, fixed_r=fixed)
    es0, es1 = O.share(bits, masked(x, bits), SEED, 70)
    e0, e1 = O.trunc_aby3(bits, k, es0, es1, SEED, 71, fixed_r=fixed)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


@pytest.mark.parametrize("bits,kx,ky", [(64, 13, 13), (64, 3, 4), (32, 6, 6)])
def test_trunc_then_mul(ctx, bits, kx, ky):
    n = 50_021
    x = W.magnitude_bounded_ints(n, bits // 2 - 3, seed=kx)
    y = W.magnitude_bounded_ints(n, bits // 2 - 3, seed=ky + 100)
    x0, x1 = _shares(ctx, bits, x, 80)
    y0, y1 = _shares(ctx, bits, y, 81)
    o0, o1 = ctx.trunc_then_mul(bits, kx, ky, x0, x1, y0, y1, tensor_id=82)
    ex0, ex1 = O.share(bits, masked(x, bits), SEED, 80)
    ey0, ey1 = O.share(bits, masked(y, bits), SEED, 81)
    e0, e1 = O.trunc_then_mul(bits, kx, ky, ex0, ex1, ey0, ey1, SEED, 82)
    assert np.array_equal(to_np(o0).astype(np.uint64), e0)
    assert np.array_equal(to_np(o1).astype(np.uint64), e1)


@pytest.mark.parametrize("op", ["drelu", "relu"])
@pytest.mark.parametrize("ring,lx,c,mag,n", [(64, 24, 0, 23, 20_011), (32, 14, 4, 17, 9_999),
                                            (32, 9, 14, 22, 4_096), (16, 5, 2, 6, 777),
                                            (64, 7, 0, 6, 1), (64, 31, 0, 32, 300)])
def test_rss_parity(ctx, op, ring, lx, c, mag, n):
    x = W.magnitude_bounded_ints(n, mag, seed=n)
    rng = np.random.default_rng(n)
    mk = np.uint64((1 << ring) - 1) if ring < 64 else np.uint64(2**64 - 1)
    x0 = rng.integers(0, 2**63, n, dtype=np.uint64) & mk
    x1 = rng.integers(0, 2**63, n, dtype=np.uint64) & mk
    x2 = (x.astype(np.uint64) - x0 - x1) & mk
    fn = ctx.rss_drelu if op == "drelu" else ctx.rss_relu
    ys = fn(Params(ring, lx, c), to_dev(x0, ring), to_dev(x1, ring), to_dev(x2, ring), tensor_id=9)
    e = O.rss_drelu(O.params(ring, lx, c), x0, x1, x2, SEED, 9, relu=(op == "relu"), threads=8)
    for g, w in zip(ys, e[:3]):
        assert np.array_equal(to_np(g).astype(np.uint64), w)


def test_rss_empty_input(ctx):
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    ys = ctx.rss_relu(Params(64, 24, 0), e, e, e, tensor_id=9)
    assert all(y.numel() == 0 for y in ys)


def test_calls_follow_torch_current_stream(ctx):
    """Calls launch on torch's current stream: a call inside torch's CUDA-graph
    capture is captured (a launch on any other stream would break the
    capture), and a call under a side-stream context matches the default one."""
    n = 5_000
    x = W.magnitude_bounded_ints(n, 23, seed=93)
    s0, s1 = _shares(ctx, 64, x, 94)
    prm = Params(64, 24, 0)
    want0, want1 = ctx.relu(prm, s0, s1, tensor_id=95)
    o0, o1 = torch.empty_like(s0), torch.empty_like(s1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.relu(prm, s0, s1, tensor_id=95, out=(o0, o1))
    side.synchronize()
    assert torch.equal(o0, want0) and torch.equal(o1, want1)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        ctx.relu(prm, s0, s1, tensor_id=95, out=(o0, o1))
    o0.zero_()
    o1.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(o0, want0) and torch.equal(o1, want1)


def test_batch_host_buffers_match_device_batch(ctx):
    """bc_relu_batch_host: the batched kernel reads and writes pinned host
    buffers across the host link; the outputs equal the device-resident
    batch's.  Tensors are slices of a few pinned arrays (and one tensor of its
    own); pageable buffers are refused before anything is launched."""
    import ctypes
    from paper_2309_04909_gb300 import BicoptorError
    from paper_2309_04909_gb300._native import BatchConfig, TensorDesc
    specs = [(64, 24, 0, 23), (32, 14, 4, 17), (64, 7, 0, 6), (16, 5, 2, 6)]
    rng = np.random.default_rng(11)
    dev_items, host_items = [], []
    for ring, lx, c, mag in specs:
        sizes = [int(v) for v in rng.integers(1, 30_000, size=5)]
        total = sum(sizes)
        x = W.magnitude_bounded_ints(total, mag, seed=ring + lx)
        s0, s1 = _shares(ctx, ring, x, 300 + lx)
        h0, h1 = s0.cpu().pin_memory(), s1.cpu().pin_memory()
        o0, o1 = ctx._empty(total, ring), ctx._empty(total, ring)
        ho0 = torch.zeros(total, dtype=o0.dtype).pin_memory()
        ho1 = torch.zeros(total, dtype=o0.dtype).pin_memory()
        off = 0
        for j, sz in enumerate(sizes):
            sl = slice(off, off + sz)
            tid, op = 400 + lx * 10 + j, j % 2
            dev_items.append((Params(ring, lx, c), s0[sl], s1[sl], o0[sl], o1[sl], tid, op))
            host_items.append((Params(ring, lx, c), h0[sl], h1[sl], ho0[sl], ho1[sl], tid, op))
            off += sz
    lone = torch.zeros(1000, dtype=torch.int64)
    lone_in = lone.pin_memory()
    lone_out0, lone_out1 = torch.zeros(1000, dtype=torch.int64).pin_memory(), \
        torch.zeros(1000, dtype=torch.int64).pin_memory()
    host_items.append((Params(64, 24, 0), lone_in, lone_in, lone_out0, lone_out1, 999))
    dz = lone.cuda()
    dev_items.append((Params(64, 24, 0), dz, dz, torch.empty_like(dz), torch.empty_like(dz), 999))
    for sched in (1, 0):
        ctx.relu_batch_plan(dev_items, schedule=sched)
        ctx.relu_batch_run()
        assert ctx.batch_status() == 0
        ctx.relu_batch_host(host_items, schedule=sched)
        for d, h in zip(dev_items, host_items):
            assert torch.equal(d[3].cpu(), h[3]) and torch.equal(d[4].cpu(), h[4])
    # a pageable buffer: the binding refuses it, and so does the C-ABI itself
    with pytest.raises(BicoptorError):
        ctx.relu_batch_host([(Params(64, 24, 0), lone, lone, lone_out0, lone_out1, 1)])
    page = np.zeros(1000, dtype=np.uint64)
    arr = (TensorDesc * 1)()
    arr[0] = TensorDesc(page.ctypes.data, page.ctypes.data, lone_out0.data_ptr(),
                        lone_out1.data_ptr(), 1000, 1, 0, Params(64, 24, 0).c_struct(), 0)
    rc = ctx._lib.bc_relu_batch_host(ctx._h, arr, 1, ctypes.byref(BatchConfig(0, 0, 0, 0, 0)))
    assert rc == -1
