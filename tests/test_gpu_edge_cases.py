"""Exhaustive and edge-case parity of every CUDA path with the oracle.

Brute force (Alg. drelu steps 1-11, Alg. relu): at l = 8 every x in Z_256
and every R in Z_256 -- the explicit shares [x]_0 = x + R, [x]_1 = -R --
each pair once at an element whose flip bit t (step 1) is 0 and once at one
whose t is 1, for (lx, c) in {(2,0), (3,0), (4,0), (3,1), (2,2)}; at l = 10
the same over Z_1024 x Z_1024 for (5,0), (4,1), (4,2).  Every output share of
every path (the single-tensor kernel, the small-launch kernel, both batched
schedules, the party-separated launches, the RSS kernel) equals the oracle's
bit for bit.  Two checks do not go through the oracle: P2's DReLU' read from
the kernel's audit equals the exact form of Thm. newtrc2 with steps 4-9 (the
masks, the shuffle and the reshare keep the zero set), and the reconstructed
DReLU equals the plaintext sign outside the exception set (reading 14 of the
paper's correctness domain: the magnitudes xi* with xi* + ceil(xi*/2) in
{2^lx - 1, 2^lx} at c = 0; also |x| < 2^c and a band around xi* 2^c at c > 0).

Edge set: at l = 64, lx = 24 the values 0, +-1, +-xi* (11,184,810), +-(xi*+1),
+-(2^24 - 1), +-2^24, +-2^47, -2^63, 2^63 - 1 with R in {0, 1, 2^64 - 1, 2^63}
and random R; at l = 32 the analogous set for (lx, c) = (9, 14) and (14, 4).
Each pair again under both flip bits, on every path including the fused
product -> truncation -> ReLU step and the audited messages.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_04909_gb300 import Context, Params
from tests._util import cuda_ok, to_dev, to_np
from tests.test_oracle_pins import _c0_exceptions, _closed_form_dprime, _predicted_miss

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

SEED = 0x5EED_00ED_6E00
THREADS = 0          # filled in at first use: all host cores


def _threads():
    global THREADS
    if not THREADS:
        THREADS = O.max_threads()
    return THREADS


@pytest.fixture(scope="module")
def ctx():
    c = Context(SEED)
    yield c
    c.close()


def _mask(ell):
    return np.uint64((1 << ell) - 1) if ell < 64 else np.uint64(2**64 - 1)


def _t_bits(tid, n):
    """Flip bit t (Alg. drelu step 1) of elements 0..n-1 of tensor `tid`: it
    depends on (seed, tid, element) only, so the oracle's audit of any input
    gives it."""
    z = np.zeros(n, np.uint64)
    _, _, aud = O.drelu(O.params(8, 2, 0), z, z, SEED, tid, audit=True, threads=_threads())
    return aud["t"]


def _both_t_layout(ell, s0, s1, tid, min_n=0, seed=0):
    """Arrays of shares in which pair j = (s0[j], s1[j]) sits at element a[j],
    whose t is 0, and at element b[j], whose t is 1.  The other elements hold
    random shares (checked too)."""
    m = s0.size
    n = max(min_n, 2 * m + 64 * int(np.sqrt(m)) + 256)
    t = _t_bits(tid, n)
    i0, i1 = np.nonzero(t == 0)[0], np.nonzero(t == 1)[0]
    assert i0.size >= m and i1.size >= m
    rng = np.random.default_rng(seed)
    a0 = rng.integers(0, 2**64, n, dtype=np.uint64) & _mask(ell)
    a1 = rng.integers(0, 2**64, n, dtype=np.uint64) & _mask(ell)
    a, b = i0[:m], i1[:m]
    a0[a], a1[a], a0[b], a1[b] = s0, s1, s0, s1
    return a0, a1, a, b, t


def _pairs(ell, xs, rs):
    """Every (x, R) of the two lists as explicit shares x + R, -R."""
    m = _mask(ell)
    X, R = np.meshgrid(np.asarray(xs, dtype=np.uint64) & m, np.asarray(rs, dtype=np.uint64) & m,
                       indexing="ij")
    X, R = X.ravel(), R.ravel()
    return X, (X + R) & m, (np.uint64(0) - R) & m


def _signed(v, ell):
    v = v.astype(np.uint64) & _mask(ell)
    if ell == 64:
        return v.view(np.int64)
    v = v.astype(np.int64)
    return np.where(v >= 1 << (ell - 1), v - (1 << ell), v)


def _eq(gpu, want):
    return np.array_equal(to_np(gpu).astype(np.uint64), want)


def _check_sign(ell, lx, c, X, rec_drelu, exhaustive):
    """The reconstructed DReLU against the plaintext sign on the domain
    |x| < 2^(lx+c), x != 0, outside the predicted exception set."""
    xs = _signed(X, ell)
    lim = 1 << (lx + c)
    dom = (xs > -lim) & (xs < lim) & (xs != 0)        # (abs() of -2^63 wraps in int64)
    bad = dom & (rec_drelu != (xs >= 0))
    mags = set(np.abs(xs[bad]).tolist())
    if exhaustive and c == 0 and lx >= 3:
        assert mags == _c0_exceptions(lx)
    else:
        assert all(_predicted_miss(v, lx, c) for v in mags), sorted(mags)[:10]


def _dprime_closed_form(ell, lx, c, s0, s1, t):
    """Thm. newtrc2 with steps 4-9 of Alg. drelu, on the flipped shares."""
    m = _mask(ell)
    neg = lambda a: (np.uint64(0) - a) & m
    fs0 = np.where(t == 1, neg(s0), s0)
    fs1 = np.where(t == 1, neg(s1), s1)
    if ell > 32:
        return _closed_form_dprime(ell, lx, c, fs0, fs1)
    # vectorised form for small rings (no overflow below 2^33)
    xp = (fs0 + fs1) & m
    rp = neg(fs1)
    mx = np.uint64((1 << lx) - 1)
    us = []
    for i in range(lx + 1):
        k1 = c + i
        lo = np.uint64((1 << k1) - 1)
        carry = ((xp & lo) + (rp & lo)) >> np.uint64(k1)
        us.append(((xp >> np.uint64(k1)) + carry) & mx)
    d = np.zeros(s0.size, dtype=bool)
    for i in range(lx + 1):
        nxt = us[i + 1] if i < lx else np.uint64(0)
        d |= ((us[i] + nxt + mx) & mx) == 0          # u_i + u_(i+1) - 1 mod 2^lx
    return d


def _all_paths(ctx, ell, lx, c, a0, a1, tid, audit=True, parties=True, rss=True):
    """Runs DReLU and ReLU on (a0, a1) through every CUDA path and compares
    each against the oracle.  Returns the oracle's DReLU shares and audit."""
    n = a0.size
    prm, P = Params(ell, lx, c), O.params(ell, lx, c)
    s0, s1 = to_dev(a0, ell), to_dev(a1, ell)
    ed0, ed1, eaud = O.drelu(P, a0, a1, SEED, tid, audit=True, threads=_threads())
    er0, er1 = O.relu(P, a0, a1, SEED, tid, threads=_threads())
    # single-tensor kernel, with and without the audit
    g0, g1 = ctx.drelu(prm, s0, s1, tensor_id=tid)
    assert _eq(g0, ed0) and _eq(g1, ed1), "drelu"
    g0, g1 = ctx.relu(prm, s0, s1, tensor_id=tid)
    assert _eq(g0, er0) and _eq(g1, er1), "relu"
    if audit:
        g0, g1, aud = ctx.drelu(prm, s0, s1, tensor_id=tid, audit=True)
        assert _eq(g0, ed0) and _eq(g1, ed1), "drelu audit"
        L = lx + 1
        assert np.array_equal(to_np(aud["w0"]).reshape(n, L), eaud["w0"])
        assert np.array_equal(to_np(aud["w1"]).reshape(n, L), eaud["w1"])
        assert np.array_equal(to_np(aud["t"]), eaud["t"])
        assert np.array_equal(to_np(aud["dprime"]), eaud["dprime"])
        # DReLU' from the kernel against Thm. newtrc2 (no oracle involved)
        want = _dprime_closed_form(ell, lx, c, a0, a1, to_np(aud["t"]).astype(np.uint64))
        assert np.array_equal(to_np(aud["dprime"]).astype(bool), want)
    # both batched schedules, DReLU and ReLU tensors in one launch
    b = [ctx._empty(n, ell) for _ in range(4)]
    items = [(prm, s0, s1, b[0], b[1], tid, 1), (prm, s0, s1, b[2], b[3], tid, 0)]
    for sched in (1, 0):
        for x in b:
            x.zero_()
        ctx.relu_batch_plan(items, schedule=sched)
        ctx.relu_batch_run()
        assert ctx.batch_status() == 0
        assert _eq(b[0], ed0) and _eq(b[1], ed1), f"batched drelu, schedule {sched}"
        assert _eq(b[2], er0) and _eq(b[3], er1), f"batched relu, schedule {sched}"
    if parties:
        g0, g1, _ = ctx.drelu_parties(prm, s0, s1, tensor_id=tid)
        assert _eq(g0, ed0) and _eq(g1, ed1), "party-separated drelu"
        g0, g1, _ = ctx.relu_parties(prm, s0, s1, tensor_id=tid)
        assert _eq(g0, er0) and _eq(g1, er1), "party-separated relu"
        assert ctx.parties_status() == 0
    if rss:
        # replicated components with x0 + x1 = [x]_0 and x2 = [x]_1: Alg. drelu2
        # runs Alg. drelu between P0 (x0 + x1) and P1 (x2)
        rng = np.random.default_rng(tid)
        x0 = rng.integers(0, 2**64, n, dtype=np.uint64) & _mask(ell)
        x1 = (a0 - x0) & _mask(ell)
        d = [to_dev(v, ell) for v in (x0, x1, a1)]
        for relu in (False, True):
            fn = ctx.rss_relu if relu else ctx.rss_drelu
            ys = fn(prm, *d, tensor_id=tid)
            e = O.rss_drelu(P, x0, x1, a1, SEED, tid, relu=relu, threads=_threads())
            for gy, wy in zip(ys, e[:3]):
                assert _eq(gy, wy), f"rss relu={relu}"
    return ed0, ed1, eaud


BRUTE = [(8, 2, 0), (8, 3, 0), (8, 4, 0), (8, 3, 1), (8, 2, 2), (10, 5, 0), (10, 4, 1), (10, 4, 2)]


@pytest.mark.parametrize("ell,lx,c", BRUTE)
def test_bruteforce_every_x_every_r_both_t(ctx, ell, lx, c):
    full = np.arange(1 << ell, dtype=np.uint64)
    X, p0, p1 = _pairs(ell, full, full)
    tid = 1000 + ell * 100 + lx * 10 + c
    a0, a1, ia, ib, t = _both_t_layout(ell, p0, p1, tid, seed=tid)
    assert (t[ia] == 0).all() and (t[ib] == 1).all()
    ed0, ed1, _ = _all_paths(ctx, ell, lx, c, a0, a1, tid)
    # the plaintext sign of every pair under both flips (through the
    # oracle-equal GPU outputs)
    rec = (ed0 + ed1) & _mask(ell)
    for pos in (ia, ib):
        _check_sign(ell, lx, c, X, rec[pos].astype(np.int64), exhaustive=True)


@pytest.mark.parametrize("ell,lx,c", BRUTE)
def test_bruteforce_small_launches(ctx, ell, lx, c):
    """The same pairs in launches small enough for the four-lanes-per-element
    kernel (every pair at l = 8, 16 random chunks of 2,048 pairs at l = 10)."""
    full = np.arange(1 << ell, dtype=np.uint64)
    X, p0, p1 = _pairs(ell, full, full)
    prm, P = Params(ell, lx, c), O.params(ell, lx, c)
    chunks = np.array_split(np.arange(X.size), X.size // 2048)
    if ell > 8:
        pick = np.random.default_rng(lx * 10 + c).choice(len(chunks), 16, replace=False)
        chunks = [chunks[i] for i in pick]
    for k, ch in enumerate(chunks):
        tid = 5000 + k
        a0, a1, _, _, _ = _both_t_layout(ell, p0[ch], p1[ch], tid, seed=k)
        assert a0.size < 10_000
        s0, s1 = to_dev(a0, ell), to_dev(a1, ell)
        for op in ("drelu", "relu"):
            g0, g1 = getattr(ctx, op)(prm, s0, s1, tensor_id=tid)
            e0, e1 = getattr(O, op)(P, a0, a1, SEED, tid, threads=_threads())
            assert _eq(g0, e0) and _eq(g1, e1), (op, k)


def _xi_star(lx):
    return sorted(_c0_exceptions(lx))


EDGE_R64 = [0, 1, 2**64 - 1, 2**63]


def _edge_values(ell, lx, c):
    xs = {0, 1, -1, (1 << (lx + c)) - 1, -((1 << (lx + c)) - 1), 1 << (lx + c),
          -(1 << (lx + c)), -(1 << (ell - 1)), (1 << (ell - 1)) - 1}
    for e in _xi_star(lx):
        for d in (0, 1, -1):
            xs |= {(e << c) + d, -((e << c) + d)}
    if c:
        xs |= {(1 << c) - 1, -((1 << c) - 1), 1 << c, -(1 << c)}
    if ell == 64:
        xs |= {1 << 47, -(1 << 47)}
    return sorted(xs)


def _edge_rs(ell, k=12):
    rng = np.random.default_rng(ell)
    m = int(_mask(ell))
    fixed = [0, 1, m, 1 << (ell - 1)]
    return fixed + [int(v) & m for v in rng.integers(0, 2**64, k, dtype=np.uint64)]


EDGE = [(64, 24, 0), (32, 9, 14), (32, 14, 4), (64, 7, 0), (64, 31, 2)]


@pytest.mark.parametrize("ell,lx,c", EDGE)
@pytest.mark.parametrize("size", ["small", "large"])
def test_edge_values(ctx, ell, lx, c, size):
    """Boundary inputs and extreme shares under both flips, alone (a small
    launch) and inside 100,000 random shares (the element-per-thread kernel)."""
    xs = _edge_values(ell, lx, c)
    X, p0, p1 = _pairs(ell, [x & int(_mask(ell)) for x in xs], _edge_rs(ell))
    tid = 7000 + ell + lx + c + (0 if size == "small" else 1)
    a0, a1, ia, ib, _ = _both_t_layout(ell, p0, p1, tid, min_n=0 if size == "small" else 100_000,
                                       seed=tid)
    ed0, ed1, eaud = _all_paths(ctx, ell, lx, c, a0, a1, tid)
    rec = (ed0 + ed1) & _mask(ell)
    for pos in (ia, ib):
        _check_sign(ell, lx, c, X, rec[pos].astype(np.int64), exhaustive=False)
    if (ell, lx, c) == (64, 24, 0):
        # xi* fails under about half of the (R, t) draws, xi* + 1 never
        xs_s = _signed(X, 64)
        d = np.concatenate([rec[ia], rec[ib]]).astype(np.int64)
        xx = np.concatenate([xs_s, xs_s])
        assert (d[np.abs(xx) == 11_184_811] == (xx[np.abs(xx) == 11_184_811] > 0)).all()
        assert (d[np.abs(xx) == 11_184_810] != (xx[np.abs(xx) == 11_184_810] > 0)).any()


def test_edge_values_fused_step(ctx):
    """The fused Beaver product -> Alg. smltrc / Alg. newtrc -> ReLU step on
    edge inputs: x from the l = 64 edge set with extreme R, y = 1.0 (f = 16)
    and y = -1.0 with random shares; all eight outputs against the oracle."""
    ell, f = 64, 16
    xs = _edge_values(64, 24, 0)
    X, x0, x1 = _pairs(ell, [x & (2**64 - 1) for x in xs], _edge_rs(64))
    n = X.size * 2
    x0, x1 = np.concatenate([x0, x0]), np.concatenate([x1, x1])
    y = np.concatenate([np.full(X.size, 1 << f, np.uint64),
                        np.full(X.size, (2**64 - (1 << f)), np.uint64)])
    y0, y1 = O.share(64, y, SEED, 3)
    prm = Params(64, 24, 0)
    for tid in (11, 12):
        w = ctx.linear_relu(64, f, prm, to_dev(x0, 64), to_dev(x1, 64), to_dev(y0, 64),
                            to_dev(y1, 64), tensor_id=tid)
        p0, p1 = O.mul_beaver(64, x0, x1, y0, y1, SEED, tid)
        t0, t1 = O.trunc_prob(64, f, p0, p1)
        d0, d1 = O.trunc_det(64, f, 0, p0, p1)
        r0, r1 = O.relu(O.params(64, 24, 0), t0, t1, SEED, tid + 1, threads=_threads())
        for name, want in (("prod0", p0), ("prod1", p1), ("trc0", t0), ("trc1", t1),
                           ("det0", d0), ("det1", d1), ("relu0", r0), ("relu1", r1)):
            assert _eq(w[name], want), (tid, name)
        assert n == w["relu0"].numel()
