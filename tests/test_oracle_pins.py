"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms derived from its theorems, exhaustive enumeration,
the plaintext it should compute, or an independent library implementation.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _mask(ell):
    return (1 << ell) - 1


# --------------------------------------------------------------------------
# Worked examples (Sec. 1 and Sec. 5.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("row", _rows("worked_examples.txt"), ids=lambda r: r[0])
def test_worked_truncation_examples(row):
    name, ell, k1, k2, alg, x, R, sh0, sh1, res, res_bits = row
    ell, k1, k2, res_bits = int(ell), int(k1), int(k2), int(res_bits)
    x, R, sh0, sh1, res = (int(v, 2) for v in (x, R, sh0, sh1, res))
    # the paper's sharing [x]_0 = x + R, [x]_1 = -R reproduces its printed shares
    assert O.share_with_r(ell, x, R) == (sh0, sh1)
    if alg == "smltrc":
        o0, o1 = O.trunc_prob(ell, k1, [sh0], [sh1])
        assert int(O.reconstruct(ell, o0, o1)[0]) == res
    else:
        o0, o1 = O.trunc_det(ell, k1, k2, [sh0], [sh1])
        assert ell - k1 - k2 == res_bits
        assert int(O.reconstruct(res_bits, o0, o1)[0]) == res


def test_cut_definition_small():
    # cut keeps bits k1..l-k2-1 and moves them to position 0 (Sec. 2.3)
    assert O.cut(0b01001011, 8, 4) == 0b0100
    assert O.cut(0b01001011, 8, 4, 1) == 0b100
    assert O.cut(0b11110101, 8, 4) == 0b1111
    for a in range(256):
        for k1 in range(8):
            for k2 in range(8 - k1):
                assert O.cut(a, 8, k1, k2) == (a >> k1) % (1 << (8 - k1 - k2))


def test_sign_table_rows():
    """Table 'sign determination' (Sec. 5.2), l=64, lx=7, x=+-22: the paper's
    value of each row is reachable for some R, and every R gives that row's
    floor(x / 2^k) or floor(x / 2^k) + 1 in Z_{2^7} (Thm. newtrc2)."""
    ell, lx = 64, 7
    rng = np.random.default_rng(5)
    R = rng.integers(0, 2**63, size=4000, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=4000, dtype=np.uint64)
    # also R whose low bits are all ones / zeros so both carries occur
    R = np.concatenate([R, np.arange(0, 256, dtype=np.uint64),
                        np.uint64(2**64 - 1) - np.arange(0, 256, dtype=np.uint64)])
    for row in _rows("sign_table.txt"):
        k = int(row[0])
        for x, printed, e0 in ((22, int(row[1], 2), int(row[2])),
                               (-22, int(row[3], 2), int(row[4]))):
            xs = np.full(R.size, x % 2**64, dtype=np.uint64)
            s0 = xs + R
            s1 = np.uint64(0) - R
            o0, o1 = O.trunc_det(ell, k, ell - lx - k, s0, s1)
            got = set(O.reconstruct(lx, o0, o1).tolist())
            base = (x >> k) % 2**lx          # floor(x / 2^k) mod 2^7
            assert got <= {base, (base + 1) % 2**lx}
            assert printed in got
            # printed e0 is the deviation from cut(xi, k) with the sign of x
            xi = abs(x)
            expect = (xi >> k) + e0 if x > 0 else -(xi >> k) + e0
            assert printed == expect % 2**lx


# --------------------------------------------------------------------------
# SecureML truncation: exact failure law (Cor. 2) and the deterministic one
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_smltrc_failure_law_exhaustive_l8(k):
    """Per Cor. 2, e1 occurs iff x + R mod 2^l < x (positive x) or
    x < x + R mod 2^l (negative x): for uniform R that is exactly |x| of the
    2^l values.  Failure = more than one away from floor(x / 2^k).  Alg.
    newtrc never fails: it gives floor(x/2^k) or floor(x/2^k)+1 mod 2^(l-k)."""
    ell, m = 8, 255
    R = np.arange(256, dtype=np.uint64)
    for x in range(-100, 101):
        xs = np.full(256, x & m, dtype=np.uint64)
        s0 = (xs + R) & np.uint64(m)
        s1 = (np.uint64(0) - R) & np.uint64(m)
        o0, o1 = O.trunc_prob(ell, k, s0, s1)
        res = O.to_signed(O.reconstruct(ell, o0, o1), ell)
        want = x >> k
        assert int((np.abs(res - want) > 1).sum()) == abs(x)
        d0, d1 = O.trunc_det(ell, k, 0, s0, s1)
        rd = set(O.reconstruct(ell - k, d0, d1).tolist())
        assert rd <= {want % 2**(ell - k), (want + 1) % 2**(ell - k)}


def test_trunc_det_closed_form_l64():
    """Thm. newtrc2 made exact: the reconstructed output of Alg. newtrc2 is
    ((x >> k1) + carry) mod 2^(l-k1-k2), carry = [x mod 2^k1 + R mod 2^k1 >= 2^k1]
    for the sharing [x]_0 = x + R, [x]_1 = -R."""
    rng = np.random.default_rng(11)
    n = 20000
    x = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    R = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    s0, s1 = x + R, np.uint64(0) - R
    for k1, k2 in ((16, 0), (16, 16), (3, 40), (0, 8), (31, 1)):
        o0, o1 = O.trunc_det(64, k1, k2, s0, s1)
        got = O.reconstruct(64 - k1 - k2, o0, o1)
        low = np.uint64((1 << k1) - 1)
        carry = ((x & low).astype(object) + (R & low).astype(object)) >= (1 << k1)
        want = ((x >> np.uint64(k1)).astype(object) + carry.astype(object)) % (1 << (64 - k1 - k2))
        assert (got.astype(object) == want).all()


def test_smltrc_failure_rate_l64_statistical():
    """At l = 64 the expected number of e1 failures is sum |x_i| / 2^64
    (exact per-element law); observed within 5 sigma.  Inputs: |x| < 2^56."""
    from paper_2309_04909_gb300 import workloads as W
    n = 1 << 19
    xs = W.magnitude_bounded_ints(n, 56, seed=1)
    x = xs.astype(np.uint64)
    s0, s1 = O.share(64, x, seed=0x1234, tid=9)
    k = 16
    o0, o1 = O.trunc_prob(64, k, s0, s1)
    res = O.to_signed(O.reconstruct(64, o0, o1), 64)
    want = xs >> k
    fails = int((np.abs(res.astype(object) - want.astype(object)) > 1).sum())
    pvec = np.abs(xs).astype(np.float64) / 2.0**64
    mu, var = pvec.sum(), (pvec * (1 - pvec)).sum()
    assert abs(fails - mu) < 5 * math.sqrt(var) + 1, (fails, mu)
    d0, d1 = O.trunc_det(64, k, 0, s0, s1)
    rd = O.reconstruct(48, d0, d1).astype(object)
    w = (want.astype(object)) % (1 << 48)
    assert (((rd - w) % (1 << 48)) <= 1).all()


# --------------------------------------------------------------------------
# Alg. modswitch: zero <-> zero, exhaustively
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lp", [1, 2, 3, 5, 8, 10])
def test_modswitch_zero_preservation_exhaustive(lp):
    a, b = np.meshgrid(np.arange(1 << lp, dtype=np.uint64), np.arange(1 << lp, dtype=np.uint64))
    a, b = a.ravel(), b.ravel()
    zero_in = ((a + b) & np.uint64((1 << lp) - 1)) == 0
    primes = [q for q in range((1 << lp) + 1, 1 << (lp + 1)) if all(q % d for d in range(2, q))][:3]
    assert primes[0] == O.prime_above(lp)
    for p in primes:
        o0, o1 = O.mod_switch(lp, p, a, b)
        assert (o0 < p).all() and (o1 < p).all()
        zero_out = ((o0.astype(np.uint64) + o1.astype(np.uint64)) % np.uint64(p)) == 0
        assert (zero_in == zero_out).all()


def test_prime_above():
    for lx in (2, 3, 4, 5, 7, 9, 14, 24):
        p = O.prime_above(lx)
        assert 2**lx < p < 2**(lx + 1)
        assert all(p % d for d in range(2, int(p ** 0.5) + 1))
        assert all(any(q % d == 0 for d in range(2, int(q ** 0.5) + 1))
                   for q in range(2**lx + 1, p))


# --------------------------------------------------------------------------
# Alg. drelu: brute force against the closed form and the plaintext sign
# --------------------------------------------------------------------------

def _closed_form_dprime(ell, lx, c, fs0, fs1):
    """DReLU' from Thm. newtrc2's exact form: reconstructed
    u_i = ((x' >> (c+i)) + carry_(c+i)) mod 2^lx with x' = fs0 + fs1 and
    R' = -fs1, v_i = u_i + u_(i+1) - 1 (v_lx = u_lx - 1); DReLU' = 1 iff some
    v_i = 0.  Masking by r != 0 in Z_p, shuffling and resharing keep the
    zero set (Alg. drelu steps 5-9)."""
    m, mx = (1 << ell) - 1, (1 << lx) - 1
    xp = (fs0.astype(object) + fs1.astype(object)) & m
    Rp = (-fs1.astype(object)) & m
    us = []
    for i in range(lx + 1):
        k1 = c + i
        carry = ((xp % (1 << k1)) + (Rp % (1 << k1))) >= (1 << k1)
        us.append(((xp >> k1) + carry.astype(object)) & mx)
    d = np.zeros(fs0.size, dtype=bool)
    for i in range(lx + 1):
        nxt = us[i + 1] if i < lx else 0
        d |= ((us[i] + nxt - 1) & mx) == 0
    return d


def _c0_exceptions(lx):
    """Magnitudes where, at c = 0, the mod-2^lx wrap of v_0 can vanish for a
    negative flipped input: xi + ceil(xi/2) in {2^lx - 1, 2^lx} (for lx = 2
    the wrap of v_1 adds xi = 3)."""
    out = set()
    for T in ((1 << lx) - 1, 1 << lx):
        for xi in range(max(1, 2 * T // 3 - 2), 2 * T // 3 + 3):
            if xi < (1 << lx) and xi + (xi + 1) // 2 == T:
                out.add(xi)
    if lx == 2:
        out.add(3)
    return out


def _predicted_miss(xi, lx, c):
    """Sign misses allowed on the domain: at c = 0 exactly the magnitudes
    above; at c > 0 also |x| < 2^c (the window skips those bits) and a band
    of half-width 2^c around each xi* 2^c."""
    if xi < (1 << c):
        return True
    return any(abs(xi - e * (1 << c)) < (1 << c) for e in _c0_exceptions(lx))


BRUTE = [(8, 2, 0), (8, 3, 0), (8, 4, 0), (8, 3, 1), (8, 2, 2), (10, 5, 0), (10, 4, 1), (10, 4, 2)]


@pytest.mark.parametrize("ell,lx,c", BRUTE)
def test_drelu_bruteforce(ell, lx, c):
    """Every x in Z_{2^l}, every R in Z_{2^l}, t in {0, 1}."""
    P = O.params(ell, lx, c)
    L, p, m = lx + 1, P.p, (1 << ell) - 1
    X, RR, T = np.meshgrid(np.arange(1 << ell, dtype=np.uint64), np.arange(1 << ell, dtype=np.uint64),
                           np.array([0, 1], dtype=np.uint64), indexing="ij")
    X, RR, T = X.ravel(), RR.ravel(), T.ravel()
    s0 = (X + RR) & np.uint64(m)
    s1 = (np.uint64(0) - RR) & np.uint64(m)
    n = X.size
    rng = np.random.default_rng(ell * 100 + lx * 10 + c)
    fy = rng.integers(0, 2**32, size=(n, L), dtype=np.uint64).astype(np.uint32)
    r = rng.integers(1, p, size=(n, L)).astype(np.uint32)
    z = rng.integers(0, p, size=(n, L)).astype(np.uint32)
    d = O.drelu_core_many(P, s0, s1, T.astype(np.uint8), fy, r, z).astype(bool)
    neg = lambda a: (np.uint64(0) - a) & np.uint64(m)
    fs0 = np.where(T == 1, neg(s0), s0)
    fs1 = np.where(T == 1, neg(s1), s1)
    assert (d == _closed_form_dprime(ell, lx, c, fs0, fs1)).all()
    # plaintext sign: DReLU = DReLU' xor t equals [x >= 0] on the domain
    # |x| < 2^(lx+c), x != 0 (DReLU(0) is irrelevant for ReLU, Sec. 5.4),
    # except on the exception set of the wrap of v_0.
    xs = X.astype(np.int64)
    xs = np.where(xs >= 1 << (ell - 1), xs - (1 << ell), xs)
    got = d.astype(np.int64) ^ T.astype(np.int64)
    dom = (np.abs(xs) < (1 << (lx + c))) & (xs != 0)
    bad = dom & (got != (xs >= 0))
    mags = set(np.abs(xs[bad]).tolist())
    if c == 0 and lx >= 3:
        assert mags == _c0_exceptions(lx)
    else:
        assert all(_predicted_miss(xi, lx, c) for xi in mags)
    if lx >= 3:
        assert bad.sum() <= 0.25 * dom.sum()


def test_drelu_exception_l64():
    """The c = 0 exception magnitude at l = 64, lx = 24: xi* = 11,184,810
    (xi + ceil(xi/2) = 2^24 - 1) fails for about half of the (R, t) draws,
    xi* + 1 never does, and random in-range inputs give the exact sign."""
    P = O.params(64, 24, 0)
    n = 600
    for xi, expect_fail in ((11184810, True), (11184811, False)):
        for sgn in (1, -1):
            x = np.full(n, (sgn * xi) % 2**64, dtype=np.uint64)
            s0, s1 = O.share(64, x, seed=77, tid=sgn + 5)
            o0, o1 = O.drelu(P, s0, s1, seed=99, tid=sgn + 5)
            got = O.reconstruct(64, o0, o1)
            fails = int((got != (1 if sgn > 0 else 0)).sum())
            if expect_fail:
                assert 0.3 * n < fails < 0.7 * n
            else:
                assert fails == 0
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(4000, 23, seed=3)
    xs = xs[np.abs(xs) != 11184810]
    xs = xs[xs != 0]
    s0, s1 = O.share(64, xs.astype(np.uint64), seed=1, tid=2)
    o0, o1 = O.drelu(P, s0, s1, seed=3, tid=2)
    assert (O.reconstruct(64, o0, o1) == (xs >= 0)).all()


def test_shuffle_moves_the_zero_uniformly():
    """Alg. drelu step 6: the shuffle is a uniform permutation, so the
    message slot k* that carries the zero of v (elements with exactly one
    zero) is uniform over the lx+1 slots, and k* equals the zero's source
    index i* (a fixed point) with probability 1/(lx+1).  i* comes from the
    closed form of Thm. newtrc2, k* from P2's view of the messages."""
    ell, lx, c = 16, 5, 0
    P = O.params(ell, lx, c)
    L, m, mx = lx + 1, (1 << ell) - 1, (1 << lx) - 1
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(60000, lx, seed=12)
    s0, s1 = O.share(ell, xs.astype(np.uint64) & np.uint64(m), seed=8, tid=1)
    o0, o1, aud = O.drelu(P, s0, s1, seed=9, tid=2, audit=True)
    t = aud["t"].astype(object)
    fs0 = np.array([(-int(a) if tt else int(a)) & m for a, tt in zip(s0, t)], dtype=object)
    fs1 = np.array([(-int(b) if tt else int(b)) & m for b, tt in zip(s1, t)], dtype=object)
    xp = (fs0 + fs1) & m
    Rp = (-fs1) & m
    u = [((xp >> i) + (((xp % (1 << i)) + (Rp % (1 << i))) >= (1 << i)).astype(object)) & mx
         for i in range(L)]
    zero = np.stack([((u[i] + (u[i + 1] if i < lx else 0) - 1) & mx) == 0 for i in range(L)], 1)
    w = (aud["w0"].astype(np.uint64) + aud["w1"].astype(np.uint64)) % np.uint64(P.p)
    one = zero.sum(1) == 1
    i_star = zero[one].argmax(1)
    k_star = (w[one] == 0).argmax(1)
    n1 = int(one.sum())
    assert n1 > 20000
    assert ((w[one] == 0).sum(1) == 1).all()
    fixed = (i_star == k_star).mean()
    assert abs(fixed - 1 / L) < 5 * math.sqrt((1 / L) * (1 - 1 / L) / n1)
    hist = np.bincount(k_star, minlength=L)
    chi2 = (((hist - n1 / L) ** 2) / (n1 / L)).sum()
    assert chi2 < 30          # 5 dof; p ~ 2e-5


def test_relu_beaver_identity():
    """Alg. relu: reconstruct(ReLU shares) = x * (DReLU' xor t) mod 2^l
    exactly (Beaver identity), and equals max(x, 0) on in-domain inputs."""
    from paper_2309_04909_gb300 import workloads as W
    for ell, lx, c, bits in ((64, 24, 0, 23), (32, 9, 14, 22), (32, 14, 4, 17), (16, 5, 2, 6)):
        P = O.params(ell, lx, c)
        xs = W.magnitude_bounded_ints(3000, bits, seed=ell + lx)
        x = xs.astype(np.uint64) & np.uint64(_mask(ell))
        s0, s1 = O.share(ell, x, seed=5, tid=1)
        o0, o1, aud = O.relu(P, s0, s1, seed=6, tid=1, audit=True)
        rec = O.reconstruct(ell, o0, o1)
        b = aud["dprime"].astype(np.uint64) ^ aud["t"].astype(np.uint64)
        want = (x.astype(object) * b.astype(object)) % (1 << ell)
        assert (rec.astype(object) == want).all()
        signed = O.to_signed(rec, ell)
        miss = np.abs(xs[signed != np.maximum(xs, 0)])
        # every miss lies in the predicted exception set of the sign test
        assert all(_predicted_miss(int(xi), lx, c) for xi in miss)
        assert miss.size < 0.08 * xs.size


def test_drelu_output_shares_and_messages():
    """Alg. drelu steps 10-11: reconstructed output is DReLU' xor t; the
    messages P2 receives reconstruct to a zero exactly when DReLU' = 1; every
    message lies in Z_p."""
    P = O.params(64, 24, 0)
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(2000, 20, seed=8)
    s0, s1 = O.share(64, xs.astype(np.uint64), seed=3, tid=4)
    o0, o1, aud = O.drelu(P, s0, s1, seed=3, tid=4, audit=True)
    rec = O.reconstruct(64, o0, o1)
    assert (rec == (aud["dprime"] ^ aud["t"])).all()
    w = (aud["w0"].astype(np.uint64) + aud["w1"].astype(np.uint64)) % np.uint64(P.p)
    assert ((w == 0).any(axis=1) == aud["dprime"].astype(bool)).all()
    assert (aud["w0"] < P.p).all() and (aud["w1"] < P.p).all()
    # step 10: P2's reply [DReLU']_1 and P0's seed02 share [DReLU']_0 add up to
    # DReLU'; step 11 unflips: o0 = t + (1-2t) d0, o1 = (1-2t) d1
    t = aud["t"].astype(object)
    sgn = [1 - 2 * v for v in t]
    d1 = aud["reply"].astype(object)
    d0 = [((int(a) - int(tt)) * s) % 2**64 for a, tt, s in zip(o0, t, sgn)]
    assert all((a + int(b)) % 2**64 == int(dp) for a, b, dp in zip(d0, d1, aud["dprime"]))
    assert all(int(b) == (int(d) * s) % 2**64 for b, d, s in zip(o1, d1, sgn))


@pytest.mark.parametrize("lx,c,p", [(31, 2, 4294967291), (31, 0, 2**31 + 11), (24, 0, 2**24 + 43)])
def test_drelu_messages_from_definition(lx, c, p):
    """Steps 1-8 of Alg. drelu recomputed with Python integers from their
    definitions (flip, windows, pair sums, modulo switch, mask, reshare) for
    explicit randomness and the identity shuffle (every Fisher-Yates word
    2^32 - 1 keeps each slot in place).  Includes p near 2^32, where the
    masked products need more than 64 bits before reduction."""
    ell = 64
    P = O.params(ell, lx, c, p=p)
    rng = np.random.default_rng(lx + c)
    M = 2**ell
    L = lx + 1
    for trial in range(40):
        x = int(rng.integers(-2**(lx + c - 1), 2**(lx + c - 1)))
        R = int(rng.integers(0, 2**63)) * 2 + trial % 2
        s0, s1 = (x + R) % M, (-R) % M
        t = trial % 2
        r = [int(v) for v in rng.integers(1, p, size=L)]
        z = [int(v) for v in rng.integers(0, p, size=L)]
        dprime, m0, m1 = O.drelu_core(P, s0, s1, t, [2**32 - 1] * lx, r, z)
        f0, f1 = ((-s0) % M, (-s1) % M) if t else (s0, s1)
        u0 = [(f0 >> (c + i)) % 2**lx for i in range(L)]
        u1 = [(-(((-f1) % M) >> (c + i))) % 2**lx for i in range(L)]
        v0 = [(u0[i] + (u0[i + 1] if i < lx else 0) - 1) % 2**lx for i in range(L)]
        v1 = [(u1[i] + (u1[i + 1] if i < lx else 0)) % 2**lx for i in range(L)]
        n0 = [a if a else 2**lx for a in v0]
        n1 = [(p + a - 2**lx) % p for a in v1]
        want0 = [(n0[k] * r[k] + z[k]) % p for k in range(L)]
        want1 = [(n1[k] * r[k] - z[k]) % p for k in range(L)]
        assert list(m0) == want0 and list(m1) == want1
        assert dprime == int(any((a + b) % p == 0 for a, b in zip(want0, want1)))


@pytest.mark.parametrize("ell,lx,c,p", [(64, 24, 0, None), (32, 14, 4, None), (64, 31, 2, 4294967291),
                                        (16, 5, 2, None)])
def test_drelu_relu_draws_from_stream_words(ell, lx, c, p):
    """Every draw of Alg. drelu / Alg. relu rebuilt with Python integers from
    the raw Philox stream words (the layout pinned in test_stream_layout):
    t and the Fisher-Yates words from seed01, rho_k = 1 + floor(W (p-1) /
    2^64) with r_k = rho_k 2^-32 mod p and z_k = floor(W' p / 2^64) from the
    slot's mask block (W, W' its two 64-bit halves, low word first), P0's
    share of DReLU' from seed02, and the ReLU triple from seed02 / seed12
    (ring elements of one word for l <= 32, two words low first above).  The
    messages, the reply and the openings of the oracle's audit must follow
    from them."""
    P = O.params(ell, lx, c, p=p)
    p = P.p
    M, L = 1 << ell, lx + 1
    seed, tid = 0x0DDB_A11_5EED, 17
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(24, min(lx + c, ell - 2), seed=lx + c)
    x = xs.astype(np.uint64) & np.uint64(_mask(ell))
    s0, s1 = O.share(ell, x, seed=9, tid=3)
    d0_, d1_, dau = O.drelu(P, s0, s1, seed=seed, tid=tid, audit=True)
    r0_, r1_, rau = O.relu(P, s0, s1, seed=seed, tid=tid, audit=True)
    inv32 = pow(2**32, -1, p)
    word = lambda pair, pur, e, j: O.stream_word(seed, pair, pur, tid, e, j)

    def ring(pair, pur, e, j):
        if ell <= 32:
            return word(pair, pur, e, j) % M
        return (word(pair, pur, e, 2 * j) | (word(pair, pur, e, 2 * j + 1) << 32)) % M

    for e in range(xs.size):
        t = word(O.PAIR_01, O.PUR_PERM, e, 0) & 1
        fy = [word(O.PAIR_01, O.PUR_PERM, e, j) for j in range(1, L)]
        r, z = [], []
        for k in range(L):
            wr = word(O.PAIR_01, O.PUR_MASK, e, 4 * k) | (word(O.PAIR_01, O.PUR_MASK, e, 4 * k + 1) << 32)
            wz = word(O.PAIR_01, O.PUR_MASK, e, 4 * k + 2) | (word(O.PAIR_01, O.PUR_MASK, e, 4 * k + 3) << 32)
            rho = 1 + ((wr * (p - 1)) >> 64)
            r.append(rho * inv32 % p)
            z.append((wz * p) >> 64)
        assert all(1 <= v < p for v in r) and all(0 <= v < p for v in z)
        dprime, m0, m1 = O.drelu_core(P, int(s0[e]), int(s1[e]), t, fy, r, z)
        assert int(dau["t"][e]) == t and int(dau["dprime"][e]) == dprime
        assert list(dau["w0"][e]) == list(m0) and list(dau["w1"][e]) == list(m1)
        assert list(rau["w0"][e]) == list(m0) and list(rau["w1"][e]) == list(m1)
        # step 10: P0's share d0 from seed02, the reply d1 = DReLU' - d0
        d0 = ring(O.PAIR_02, O.PUR_REPLY, e, 0)
        assert int(dau["reply"][e]) == (dprime - d0) % M
        sg = 1 - 2 * t
        assert int(d0_[e]) == (t + sg * d0) % M and int(d1_[e]) == (sg * (dprime - d0)) % M
        # Alg. relu: a0, b0, c0 from seed02, a1, b1 from seed12
        a0, b0, c0 = (ring(O.PAIR_02, O.PUR_RELU_TRIPLE, e, j) for j in range(3))
        a1, b1 = (ring(O.PAIR_12, O.PUR_RELU_TRIPLE, e, j) for j in range(2))
        assert int(rau["open0"][e]) == (int(s0[e]) - a0) % M
        assert int(rau["open1"][e]) == (int(s1[e]) - a1) % M
        assert int(rau["pre_c1"][e]) == ((a0 + a1) * (b0 + b1) - c0) % M
        assert int(rau["reply"][e]) == (dprime - b0 - b1) % M


def test_drelu_shuffle_from_definition():
    """Step 6 with explicit Fisher-Yates words: starting from the identity,
    step j = lx, ..., 1 takes the next word W (words consumed in order) and
    swaps positions j and floor(W (j + 1) / 2^32); message slot k then
    carries the masked window of index perm[k].  Recomputed with Python
    integers and checked against the oracle's messages."""
    ell, lx, c = 64, 24, 0
    P = O.params(ell, lx, c)
    p, M, L = P.p, 1 << ell, lx + 1
    rng = np.random.default_rng(11)
    for trial in range(30):
        x = int(rng.integers(-2**22, 2**22))
        R = int(rng.integers(0, 2**63)) * 2 + trial % 2
        s0, s1 = (x + R) % M, (-R) % M
        t = trial % 2
        fy = [int(v) for v in rng.integers(0, 2**32, size=lx, dtype=np.uint64)]
        r = [int(v) for v in rng.integers(1, p, size=L)]
        z = [int(v) for v in rng.integers(0, p, size=L)]
        dprime, m0, m1 = O.drelu_core(P, s0, s1, t, fy, r, z)
        perm = list(range(L))
        for step, j in enumerate(range(lx, 0, -1)):
            q = (fy[step] * (j + 1)) >> 32
            perm[j], perm[q] = perm[q], perm[j]
        f0, f1 = ((-s0) % M, (-s1) % M) if t else (s0, s1)
        u0 = [(f0 >> (c + i)) % 2**lx for i in range(L)]
        u1 = [(-(((-f1) % M) >> (c + i))) % 2**lx for i in range(L)]
        v0 = [(u0[i] + (u0[i + 1] if i < lx else 0) - 1) % 2**lx for i in range(L)]
        v1 = [(u1[i] + (u1[i + 1] if i < lx else 0)) % 2**lx for i in range(L)]
        n0 = [a if a else 2**lx for a in v0]
        n1 = [(p + a - 2**lx) % p for a in v1]
        want0 = [(n0[perm[k]] * r[k] + z[k]) % p for k in range(L)]
        want1 = [(n1[perm[k]] * r[k] - z[k]) % p for k in range(L)]
        assert list(m0) == want0 and list(m1) == want1
        assert dprime == int(any((a + b) % p == 0 for a, b in zip(want0, want1)))


def test_beaver_mul_exact():
    from paper_2309_04909_gb300 import workloads as W
    for ell in (64, 32, 8):
        x = W.magnitude_bounded_ints(5000, min(ell - 2, 40), seed=ell).astype(np.uint64)
        y = W.magnitude_bounded_ints(5000, min(ell - 2, 40), seed=ell + 1).astype(np.uint64)
        mk = np.uint64(_mask(ell))
        x &= mk
        y &= mk
        x0, x1 = O.share(ell, x, seed=21, tid=1)
        y0, y1 = O.share(ell, y, seed=21, tid=2)
        o0, o1 = O.mul_beaver(ell, x0, x1, y0, y1, seed=22, tid=3)
        want = (x.astype(object) * y.astype(object)) % (1 << ell)
        assert (O.reconstruct(ell, o0, o1).astype(object) == want).all()


def test_share_reconstruct_and_uniformity():
    x = np.arange(1000, dtype=np.uint64)
    for ell in (8, 32, 64):
        xm = x & np.uint64(_mask(ell))
        s0, s1 = O.share(ell, xm, seed=3, tid=7)
        assert (O.reconstruct(ell, s0, s1) == xm).all()
        assert (s0 <= np.uint64(_mask(ell))).all() and (s1 <= np.uint64(_mask(ell))).all()
    # [x]_1 = -R is uniform: byte histogram of 2^16 shares is flat (chi^2)
    s0, s1 = O.share(64, np.zeros(1 << 16, np.uint64), seed=4, tid=1)
    hist = np.bincount((s1 & np.uint64(255)).astype(np.int64), minlength=256)
    chi2 = ((hist - 256.0) ** 2 / 256.0).sum()
    assert chi2 < 400  # 255 dof; p ~ 1e-8


@pytest.mark.parametrize("ell", [64, 32, 13])
def test_share_and_beaver_shares_from_stream_words(ell):
    """The dealer's R and the Beaver product's triple rebuilt with Python
    integers from the raw stream words (ring elements of one word for
    l <= 32, two words low first above): [x]_0 = x + R, [x]_1 = -R, and the
    product's output shares [xy]_0 = de + d b0 + e a0 + c0 (de added by P0),
    [xy]_1 = d b1 + e a1 + c1 with c1 = (a0 + a1)(b0 + b1) - c0, d and e the
    openings of x - a and y - b."""
    M = 1 << ell
    seed = 0xBEA5_E4ED
    word = lambda pair, pur, tid, e, j: O.stream_word(seed, pair, pur, tid, e, j)

    def ring(pair, pur, tid, e, j):
        if ell <= 32:
            return word(pair, pur, tid, e, j) % M
        return (word(pair, pur, tid, e, 2 * j) | (word(pair, pur, tid, e, 2 * j + 1) << 32)) % M

    rng = np.random.default_rng(ell)
    x = rng.integers(0, 2**62, size=40, dtype=np.uint64) & np.uint64(_mask(ell))
    y = rng.integers(0, 2**62, size=40, dtype=np.uint64) & np.uint64(_mask(ell))
    x0, x1 = O.share(ell, x, seed=seed, tid=5)
    y0, y1 = O.share(ell, y, seed=seed, tid=6)
    o0, o1 = O.mul_beaver(ell, x0, x1, y0, y1, seed=seed, tid=9)
    for e in range(x.size):
        R = ring(O.PAIR_DEALER, O.PUR_SHARE, 5, e, 0)
        assert int(x0[e]) == (int(x[e]) + R) % M and int(x1[e]) == (-R) % M
        a0, b0, c0 = (ring(O.PAIR_02, O.PUR_MUL_TRIPLE, 9, e, j) for j in range(3))
        a1, b1 = (ring(O.PAIR_12, O.PUR_MUL_TRIPLE, 9, e, j) for j in range(2))
        c1 = ((a0 + a1) * (b0 + b1) - c0) % M
        d = (int(x0[e]) - a0 + int(x1[e]) - a1) % M
        ee = (int(y0[e]) - b0 + int(y1[e]) - b1) % M
        assert int(o0[e]) == (d * ee + d * b0 + ee * a0 + c0) % M
        assert int(o1[e]) == (d * b1 + ee * a1 + c1) % M


@pytest.mark.parametrize("ell,k,fixed_r", [(64, 16, 0), (64, 26, 1 << 26), (32, 12, 0)])
def test_aby3_from_stream_words(ell, k, fixed_r):
    """Alg. aby3trc with its preprocessing rebuilt from the raw stream words
    ([r]_0 and [r']_0 from seed02, [r]_1 from seed12, or fixed_r - [r]_0) and
    every step recomputed with Python integers: r' = r / 2^k (signed floor),
    [r']_1 = r' - [r']_0 from P2, the opened alpha = x + r, P0 keeps
    alpha / 2^k - [r']_0 and P1 -[r']_1."""
    M = 1 << ell
    seed, tid = 0xAB_3AB3, 4

    def ring(pair, e, j):
        w = lambda jj: O.stream_word(seed, pair, O.PUR_ABY3, tid, e, jj)
        return w(j) % M if ell <= 32 else (w(2 * j) | (w(2 * j + 1) << 32)) % M

    def sdiv(a):   # floor division of the signed value by 2^k, mod 2^l
        v = a - M if a >> (ell - 1) else a
        return (v >> k) % M

    rng = np.random.default_rng(k)
    x = rng.integers(0, 2**62, size=40, dtype=np.uint64) & np.uint64(_mask(ell))
    s0, s1 = O.share(ell, x, seed=seed, tid=2)
    o0, o1 = O.trunc_aby3(ell, k, s0, s1, seed, tid, fixed_r=fixed_r)
    for e in range(x.size):
        r0, rp0 = ring(O.PAIR_02, e, 0), ring(O.PAIR_02, e, 1)
        r1 = (fixed_r - r0) % M if fixed_r else ring(O.PAIR_12, e, 0)
        rp1 = (sdiv((r0 + r1) % M) - rp0) % M
        alpha = (int(s0[e]) + r0 + int(s1[e]) + r1) % M
        assert int(o0[e]) == (sdiv(alpha) - rp0) % M and int(o1[e]) == (-rp1) % M


def test_encode_round_half_even():
    f = 4
    x = np.array([0.0, 1.0, -1.0, 0.5 / 16, 1.5 / 16, 2.5 / 16, -0.5 / 16, -1.5 / 16, 3.03125])
    got = O.to_signed(O.encode(x, f, 32), 32)
    assert got.tolist() == [0, 16, -16, 0, 2, 2, 0, -2, 48]
    assert O.encode(np.array([-1.0]), 16, 64)[0] == np.uint64(2**64 - 2**16)


# --------------------------------------------------------------------------
# Philox-4x32-10 against an independent library implementation
# --------------------------------------------------------------------------

def test_philox_matches_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(2)
    rows = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64).tolist()
    rows += [[0] * 6, [2**32 - 1] * 6, [1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 1, 0]]
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, os.path.join(HERE, "philox_library_ref.py")],
                          input=json.dumps(rows), capture_output=True, text=True, env=env,
                          timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout)
    for row, want in zip(rows, ref):
        assert O.philox(row[:4], row[4:]) == want


def test_stream_layout():
    # word j of a stream is word j % 4 of block j / 4 of the documented counter
    seed, pair, pur, tid, elem = 0x0123456789ABCDEF, O.PAIR_01, O.PUR_MASK, 7, (5 << 32) | 9
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(9):
        ctr = [elem & 0xFFFFFFFF, tid, j // 4, (pair << 24) | (pur << 16) | (elem >> 32)]
        assert O.stream_word(seed, pair, pur, tid, elem, j) == O.philox(ctr, key)[j % 4]


# --------------------------------------------------------------------------
# Alg. aby3trc and Alg. linear (Sec. 2.4, Sec. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_aby3_failure_law_exhaustive_l8(k):
    """Sec. 3: ABY3 truncation fails (e1) exactly when alpha = x + r leaves
    the signed range, i.e. for |x| of the 2^l values of r."""
    for x in range(-100, 101):
        fails = 0
        for r in range(256):
            r0 = (r * 37 + 11) & 255           # any split of r works
            s0, s1 = O.share_with_r(8, x & 255, (r * 91 + 5) & 255)
            o0, o1 = O.aby3_core(8, k, s0, s1, r0, (r - r0) & 255, (r * 13) & 255)
            res = (o0 + o1) & 255
            res = res - 256 if res >= 128 else res
            fails += abs(res - (x >> k)) > 1
        assert fails == abs(x), (x, k, fails)


def test_aby3_fixed_r_hides_e1_and_random_r_does_not():
    """Sec. 4.1: with r fixed to 2^26 no e1 occurs for |x| < 2^62 (the
    implementation shortcut that hid the error); with uniform r the failure
    count matches sum |x| / 2^64 (within 5 sigma)."""
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(1 << 18, 62, seed=26)
    x = xs.astype(np.uint64)
    s0, s1 = O.share(64, x, seed=3, tid=1)
    want = xs >> 26
    for fixed, expect_zero in ((1 << 26, True), (0, False)):
        o0, o1 = O.trunc_aby3(64, 26, s0, s1, seed=4, tid=2, fixed_r=fixed)
        res = O.to_signed(O.reconstruct(64, o0, o1), 64)
        fails = int((np.abs(res.astype(object) - want.astype(object)) > 1).sum())
        if expect_zero:
            assert fails == 0
        else:
            p = np.abs(xs).astype(np.float64) / 2.0 ** 64
            assert abs(fails - p.sum()) < 5 * math.sqrt((p * (1 - p)).sum()) + 1
            assert fails > 1000


@pytest.mark.parametrize("f", [26, 25])
def test_truncate_then_multiply_exact_composition(f):
    """Alg. linear: shares reconstruct to trc(x, kx) * trc(y, ky) where each
    truncation is Alg. smltrc's (the Beaver product is exact), and the result
    stays within (|x| + |y|) / 2^(f/2) + 1 of x y / 2^f for in-range inputs,
    where multiply-then-truncate at l = 64 with f = 26 fails often.  An odd f
    splits the truncation unevenly (Sec. 4.2), so kx and ky differ."""
    from paper_2309_04909_gb300 import workloads as W
    X = W.gaussian_reals(20000, 4.0, seed=5, stream=0)
    Y = W.gaussian_reals(20000, 4.0, seed=5, stream=1)
    xi = np.rint(np.ldexp(X, f)).astype(np.int64)
    yi = np.rint(np.ldexp(Y, f)).astype(np.int64)
    x0, x1 = O.share(64, xi.astype(np.uint64), seed=6, tid=1)
    y0, y1 = O.share(64, yi.astype(np.uint64), seed=6, tid=2)
    kx, ky = f // 2, f - f // 2
    o0, o1 = O.trunc_then_mul(64, kx, ky, x0, x1, y0, y1, seed=7, tid=3)
    tx0, tx1 = O.trunc_prob(64, kx, x0, x1)
    ty0, ty1 = O.trunc_prob(64, ky, y0, y1)
    tx = O.to_signed(O.reconstruct(64, tx0, tx1), 64).astype(object)
    ty = O.to_signed(O.reconstruct(64, ty0, ty1), 64).astype(object)
    got = O.to_signed(O.reconstruct(64, o0, o1), 64).astype(object)
    assert (got == (tx * ty)).all() or all(((g - a * b) % 2**64) == 0 for g, a, b in zip(got, tx, ty))
    exact = [(int(a) * int(b)) / 2.0 ** f for a, b in zip(xi, yi)]
    bound = [(abs(int(a)) + abs(int(b))) / 2.0 ** (f // 2) + 2 for a, b in zip(xi, yi)]
    assert all(abs(float(g) - e) <= bd for g, e, bd in zip(got, exact, bound))


# --------------------------------------------------------------------------
# Alg. drelu2 (RSS) and the RSS ReLU
# --------------------------------------------------------------------------

def test_rss_drelu_bruteforce_l8():
    """Every x in Z_{2^8}, 24 replicated splits each: the three output
    components reconstruct to DReLU' xor t, DReLU' is Thm. newtrc2's closed
    form on x = x0 + x1 + x2 split as (x0 + x1, x2), and the sign is right
    outside the exception set (lx = 4, c = 0: xi* = 10)."""
    ell, lx, c, m = 8, 4, 0, 255
    P = O.params(ell, lx, c)
    rng = np.random.default_rng(9)
    X = np.repeat(np.arange(256, dtype=np.uint64), 24)
    a = rng.integers(0, 256, X.size, dtype=np.uint64)
    b = rng.integers(0, 256, X.size, dtype=np.uint64)
    x0, x1, x2 = a, b, (X - a - b) & np.uint64(m)
    seed, tid = 11, 3
    y0, y1, y2, dp = O.rss_drelu(P, x0, x1, x2, seed, tid)
    t = np.array([O.stream_word(seed, O.PAIR_01, O.PUR_PERM, tid, e, 0) & 1 for e in range(X.size)],
                 dtype=np.uint64)
    rec = (y0 + y1 + y2) & np.uint64(m)
    assert (rec == (dp.astype(np.uint64) ^ t)).all()
    # DReLU' on the 2-of-2 split (x0 + x1, x2) after the flip by t
    s0 = (x0 + x1) & np.uint64(m)
    neg = lambda v: (np.uint64(0) - v) & np.uint64(m)
    fs0, fs1 = np.where(t == 1, neg(s0), s0), np.where(t == 1, neg(x2), x2)
    assert (dp.astype(bool) == _closed_form_dprime(ell, lx, c, fs0, fs1)).all()
    xs = np.where(X >= 128, X.astype(np.int64) - 256, X.astype(np.int64))
    dom = (np.abs(xs) < 16) & (xs != 0)
    bad = dom & (rec != (xs >= 0))
    assert set(np.abs(xs[bad]).tolist()) <= _c0_exceptions(lx)


@pytest.mark.parametrize("relu", [False, True])
def test_rss_components_from_stream_words(relu):
    """Alg. drelu2 / the RSS ReLU with every preprocessing draw rebuilt from
    the raw stream words and each step recomputed with Python integers: [t]
    from alpha_0..2 (seed012) as (a0 - a2, a1 - a0 + t, a2 - a1); s from seed2
    with [s]_1 from seed012, [s]_2 from seed12 and [s]_0 = s - [s]_1 - [s]_2;
    the replicated product [s][t] with the zero sharing gamma (seed012);
    [s xor t] = [s] + [t] - 2[s][t]; the output d'' + [s xor t] - 2 d'' [s xor
    t] with d'' = s xor DReLU' added to component 0; for ReLU the replicated
    product with x and its own zero sharing."""
    ell, lx, c = 64, 24, 0
    P = O.params(ell, lx, c)
    M = 1 << ell
    seed, tid = 0x355_0DD5, 12
    rng = np.random.default_rng(23)
    x = rng.integers(-2**22, 2**22, size=30)
    xu = [int(v) % M for v in x]
    a = [int(v) for v in rng.integers(0, 2**63, size=30)]
    b = [int(v) for v in rng.integers(0, 2**63, size=30)]
    x0 = np.array(a, dtype=np.uint64)
    x1 = np.array(b, dtype=np.uint64)
    x2 = np.array([(v - u - w) % M for v, u, w in zip(xu, a, b)], dtype=np.uint64)
    y0, y1, y2, dp = O.rss_drelu(P, x0, x1, x2, seed, tid, relu=relu)

    def ring(pair, pur, e, j):
        w = lambda jj: O.stream_word(seed, pair, pur, tid, e, jj)
        return (w(2 * j) | (w(2 * j + 1) << 32)) % M

    def rmul(u, v, g):   # replicated product: component i from (i, i + 1)
        return [(u[i] * v[i] + u[i] * v[(i + 1) % 3] + u[(i + 1) % 3] * v[i] + g[i]
                 - g[(i + 1) % 3]) % M for i in range(3)]

    for e in range(x.size):
        t = O.stream_word(seed, O.PAIR_01, O.PUR_PERM, tid, e, 0) & 1
        al = [ring(O.PAIR_012, O.PUR_RSS_T, e, j) for j in range(3)]
        T = [(al[0] - al[2]) % M, (al[1] - al[0] + t) % M, (al[2] - al[1]) % M]
        s = O.stream_word(seed, O.PAIR_2, O.PUR_RSS_S, tid, e, 0) & 1
        S1, S2 = ring(O.PAIR_012, O.PUR_RSS_S, e, 0), ring(O.PAIR_12, O.PUR_RSS_S, e, 0)
        S = [(s - S1 - S2) % M, S1, S2]
        g = [ring(O.PAIR_012, O.PUR_RSS_Z, e, j) for j in range(3)]
        ST = rmul(S, T, g)
        X = [(S[j] + T[j] - 2 * ST[j]) % M for j in range(3)]
        dd = s ^ int(dp[e])
        Y = [(X[j] - 2 * dd * X[j] + (dd if j == 0 else 0)) % M for j in range(3)]
        if relu:
            gr = [ring(O.PAIR_012, O.PUR_RSS_ZR, e, j) for j in range(3)]
            Y = rmul([int(x0[e]), int(x1[e]), int(x2[e])], Y, gr)
        assert [int(y0[e]), int(y1[e]), int(y2[e])] == Y


def test_rss_relu_exact_product():
    from paper_2309_04909_gb300 import workloads as W
    for ell, lx, c, bits in ((64, 24, 0, 23), (32, 14, 4, 17)):
        P = O.params(ell, lx, c)
        mk = np.uint64((1 << ell) - 1)
        xs = W.magnitude_bounded_ints(4000, bits, seed=ell)
        rng = np.random.default_rng(ell)
        x0 = rng.integers(0, 2**63, xs.size, dtype=np.uint64) & mk
        x1 = rng.integers(0, 2**63, xs.size, dtype=np.uint64) & mk
        x2 = (xs.astype(np.uint64) - x0 - x1) & mk
        d0, d1, d2, dp = O.rss_drelu(P, x0, x1, x2, 4, 5)
        r0, r1, r2, dp2 = O.rss_drelu(P, x0, x1, x2, 4, 5, relu=True)
        assert (dp == dp2).all()
        b = ((d0 + d1 + d2) & mk).astype(object)
        rec = ((r0 + r1 + r2) & mk).astype(object)
        assert (rec == (xs.astype(object) * b) % (1 << ell)).all()
        signed = O.to_signed((r0 + r1 + r2) & mk, ell)
        miss = np.abs(xs[signed != np.maximum(xs, 0)])
        assert all(_predicted_miss(int(v), lx, c) for v in miss)


# ---- the Bicoptor 1.0-style DReLU (the baseline the paper improves on) ----------

def _smltrc_ints(ell, s0, s1, k):
    """Alg. smltrc of each party's share, from its definition (Python ints):
    P0 cut([x]_0, k), P1 2^l - cut(2^l - [x]_1, k), both mod 2^l."""
    m = (1 << ell) - 1
    return (s0 >> k) & m, (-(((-s1) & m) >> k)) & m


def _b1_closed_form(ell, lx, c, fs0, fs1):
    """DReLU' of the 1.0-style protocol from its definition: some recursive
    sum S_i = sum_{k=i..lx} trc(x', c + k), reconstructed, equals 1 (the
    masks are units, the shuffle and the reshare keep the zero set)."""
    m = (1 << ell) - 1
    out = []
    for a, b in zip(fs0.tolist(), fs1.tolist()):
        u = [sum(_smltrc_ints(ell, a, b, c + k)) & m for k in range(lx + 1)]
        out.append(any(((sum(u[i:]) - 1) & m) == 0 for i in range(lx + 1)))
    return np.array(out)


B1_BRUTE = [(8, 2, 0), (8, 3, 0), (8, 4, 0), (8, 3, 1), (8, 2, 2), (10, 5, 0), (10, 4, 2)]


@pytest.mark.parametrize("ell,lx,c", B1_BRUTE)
def test_b1_bruteforce(ell, lx, c):
    """Every x, every R, t in {0, 1}: DReLU' equals the closed form, and a
    sign is wrong only where one of the SecureML truncations makes its large
    error e1 (|trc(x', k) - floor(x' / 2^k)| > 1, probability |x| / 2^l each,
    Cor. 2) or, with key offset c > 0, for |x| < 2^c.  That is the failure
    Bicoptor 2.0's deterministic truncation removes."""
    m = (1 << ell) - 1
    L = lx + 1
    X, RR, T = np.meshgrid(np.arange(1 << ell, dtype=np.uint64),
                           np.arange(1 << ell, dtype=np.uint64),
                           np.array([0, 1], dtype=np.uint64), indexing="ij")
    X, RR, T = X.ravel(), RR.ravel(), T.ravel()
    s0 = (X + RR) & np.uint64(m)
    s1 = (np.uint64(0) - RR) & np.uint64(m)
    n = X.size
    rng = np.random.default_rng(ell * 1000 + lx * 10 + c)
    fy = rng.integers(0, 2**32, size=(n, L), dtype=np.uint64).astype(np.uint32)
    r = (rng.integers(0, 2**63, size=(n, L), dtype=np.uint64) * np.uint64(2) + np.uint64(1)) \
        & np.uint64(m)
    z = rng.integers(0, 2**63, size=(n, L), dtype=np.uint64) & np.uint64(m)
    P = O.params(ell, lx, c)
    d = O.drelu_b1_core_many(P, s0, s1, T.astype(np.uint8), fy, r, z).astype(bool)
    neg = lambda a: (np.uint64(0) - a) & np.uint64(m)
    fs0 = np.where(T == 1, neg(s0), s0)
    fs1 = np.where(T == 1, neg(s1), s1)
    assert (d == _b1_closed_form(ell, lx, c, fs0, fs1)).all()
    xs = X.astype(np.int64)
    xs = np.where(xs >= 1 << (ell - 1), xs - (1 << ell), xs)
    xp = ((fs0 + fs1) & np.uint64(m)).astype(np.int64)
    xp = np.where(xp >= 1 << (ell - 1), xp - (1 << ell), xp)
    e1 = np.zeros(n, dtype=bool)
    for k in range(lx + 1):
        a, b = _smltrc_ints(ell, fs0.astype(object), fs1.astype(object), c + k)
        uk = ((a + b) & m).astype(np.int64)
        uk = np.where(uk >= 1 << (ell - 1), uk - (1 << ell), uk)
        e1 |= np.abs(uk - (xp >> (c + k))) > 1
    got = d.astype(np.int64) ^ T.astype(np.int64)
    dom = (np.abs(xs) < (1 << (lx + c))) & (xs != 0)
    bad = dom & (got != (xs >= 0))
    above = np.abs(xs) >= (1 << c)
    assert not (bad & ~e1 & above).any()
    assert bad.sum() > 0 and (bad & above).sum() <= (e1 & dom).sum()


def test_b1_messages_recomputed():
    """The messages of the 1.0-style protocol recomputed with Python ints
    from the oracle's Philox stream words: t and the shuffle, then for every
    slot k w0 = (S0_{perm k} - 1) r_k + z_k and w1 = S1_{perm k} r_k - z_k in
    Z_{2^l}, with r_k the odd unit and z_k the reshare of slot k."""
    seed, tid = 0xB1B1, 9
    for ell, lx, c in ((64, 24, 0), (64, 7, 24), (32, 14, 4)):
        m = (1 << ell) - 1
        P = O.params(ell, lx, c)
        rng = np.random.default_rng(ell + lx)
        x = rng.integers(-(1 << (lx + c - 1)), 1 << (lx + c - 1), size=40)
        s0, s1 = O.share(ell, (x.astype(np.uint64) & np.uint64(m)), seed, 1)
        o0, o1, w0, w1, dp = O.b1(P, s0, s1, seed, tid, msgs=True)
        L = lx + 1
        for e in range(x.size):
            word = lambda pur, j: O.stream_word(seed, O.PAIR_01, pur, tid, e, j)
            t = word(O.PUR_PERM, 0) & 1
            a, b = int(s0[e]), int(s1[e])
            if t:
                a, b = (-a) & m, (-b) & m
            perm = list(range(L))
            for j in range(lx, 0, -1):
                q = (word(O.PUR_PERM, lx - j + 1) * (j + 1)) >> 32
                perm[j], perm[q] = perm[q], perm[j]
            u = [_smltrc_ints(ell, a, b, c + k) for k in range(L)]
            S0 = [sum(u0 for u0, _ in u[i:]) & m for i in range(L)]
            S1 = [sum(u1 for _, u1 in u[i:]) & m for i in range(L)]
            for k in range(L):
                w64 = lambda j: word(O.PUR_B1_MASK, 4 * k + j) | (word(O.PUR_B1_MASK, 4 * k + j + 1) << 32)
                rk, zk = (w64(0) | 1) & m, w64(2) & m
                assert int(w0[e, k]) == ((S0[perm[k]] - 1) * rk + zk) & m
                assert int(w1[e, k]) == (S1[perm[k]] * rk - zk) & m
            assert int(dp[e]) == int(any(((int(w0[e, k]) + int(w1[e, k])) & m) == 0
                                         for k in range(L)))


def test_b1_sign_at_l64():
    """At l = 64 a SecureML failure has probability |x| / 2^64 per
    truncation, so for |x| < 2^23 the 1.0-style DReLU gives the exact sign
    and its ReLU is exactly max(x, 0) (x = 0 aside)."""
    P = O.params(64, 24, 0)
    from paper_2309_04909_gb300 import workloads as W
    xs = W.magnitude_bounded_ints(20000, 23, seed=5)
    xs = xs[xs != 0]
    s0, s1 = O.share(64, xs.astype(np.uint64), seed=1, tid=2)
    o0, o1 = O.b1(P, s0, s1, 3, 4, threads=8)
    assert (O.reconstruct(64, o0, o1) == (xs >= 0)).all()
    r0, r1 = O.b1(P, s0, s1, 3, 4, relu=True, threads=8)
    assert (O.to_signed(O.reconstruct(64, r0, r1), 64) == np.maximum(xs, 0)).all()
