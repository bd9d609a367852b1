/*
 * Bicoptor 2.0 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, step-by-step CPU implementation of what the GPU hot path
 * computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code with the
 * CUDA sources.
 *
 * Paper: "Bicoptor 2.0: Addressing Challenges in Probabilistic Truncation for
 * Enhanced Privacy-Preserving Machine Learning" (arXiv 2309.04909).
 *
 * Every ring value is held in a uint64_t and reduced explicitly; every Z_p
 * value in a uint32_t (p < 2^32).  There is no floating point on the protocol
 * path; the fixed-point encoder is the only place a double appears.
 *
 * Readings of the paper that this file takes (the paper is silent or
 * ambiguous there) are marked "READING".  The pseudorandom layout (Philox
 * counters, how words become ring/Z_p elements, the Fisher-Yates rule) is not
 * in the paper at all; it is this project's fixed convention and is described
 * next to orc_stream_word below.
 *
 * Pins (tests/test_oracle_pins.py): the paper's worked 8-bit truncation
 * examples (Sec. 1, Sec. 5.1), Table "sign determination" rows, the exact
 * SecureML failure law derived from Cor. 2, exhaustive zero-preservation of
 * Alg. modswitch, brute force of Alg. drelu at l=8 and l=10 against the
 * closed form of Thm. "newtrc2" and the plaintext sign, the Beaver identity of
 * Alg. relu, and Philox-4x32-10 against an independent library implementation.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* Element-parallel loops.  Every elementwise loop of this file runs its
 * iterations independently (each element reads only its own inputs and its
 * own Philox counters), so OpenMP splits them over the host cores without
 * changing any value.  orc_set_threads(0) = OpenMP's default (all cores);
 * orc_set_threads(1) runs everything on one core.  Small loops stay serial.
 * orc_drelu, orc_relu and orc_rss_drelu take their thread count as an
 * argument instead. */
static int g_threads = 0;
void orc_set_threads(int t) { g_threads = t > 0 ? t : 0; }
#ifdef _OPENMP
static int orc_threads(void) { return g_threads > 0 ? g_threads : omp_get_max_threads(); }
#define ORC_PARALLEL_FOR \
    _Pragma("omp parallel for schedule(static) num_threads(orc_threads()) if(n >= 4096)")
#else
#define ORC_PARALLEL_FOR
#endif

/* ------------------------------------------------------------------------- */
/* Ring Z_{2^l}                                                              */
/* ------------------------------------------------------------------------- */

static uint64_t ring_mask(int ell) { return ell >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << ell) - 1); }
static uint64_t rmod(uint64_t a, int ell) { return a & ring_mask(ell); }
static uint64_t rneg(uint64_t a, int ell) { return rmod((uint64_t)0 - a, ell); }

/* Sec. 2.3: cut(alpha, k1, k2) keeps bits k1 .. l-k2-1 of alpha.
 * READING: the bits are moved down to position 0 (cut is a right shift): the
 * worked examples of Sec. 1 and cut(2^l, k) = 2^(l-k) in Sec. 5.1 need it,
 * although the displayed sum keeps the weights 2^i.  Written bit by bit,
 * exactly as the definition reads. */
uint64_t orc_cut(uint64_t alpha, int ell, int k1, int k2)
{
    uint64_t out = 0;
    for (int i = k1; i <= ell - k2 - 1; i++) {
        uint64_t bit = (alpha >> i) & 1u;
        out |= bit << (i - k1);
    }
    return out;
}

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC 2011): 10 rounds of the 4x32 S-box with the          */
/* published multipliers and Weyl key increments.                            */
/* ------------------------------------------------------------------------- */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Pre-shared seeds (Sec. 2.1): seed01, seed02, seed12.  The simulation      */
/* derives every pair's stream from one 64-bit seed, keyed by a pair tag.    */
/*                                                                           */
/* Layout (this project's convention; the paper does not specify a PRG):     */
/*   key     = (lo32(seed), hi32(seed))                                      */
/*   counter = (lo32(elem), tensor_id, block,                                */
/*              pair << 24 | purpose << 16 | (elem >> 32) & 0xffff)          */
/* Word j of a stream is word j % 4 of block j / 4.                          */
/* ------------------------------------------------------------------------- */

enum { PAIR_01 = 0x01, PAIR_02 = 0x02, PAIR_12 = 0x12, PAIR_DEALER = 0xDE,
       PAIR_012 = 0x03 /* seed012, all three parties */, PAIR_2 = 0x20 /* seed2, P2 alone */ };
enum {
    PUR_SHARE = 1,      /* dealer's R for the 2-of-2 sharing            */
    PUR_PERM = 2,       /* seed01: flip bit t and the shuffle           */
    PUR_MASK = 3,       /* seed01: r_k, z_k of message slot k           */
    PUR_REPLY = 4,      /* seed02: P0's share of DReLU'                 */
    PUR_RELU_TRIPLE = 5,/* seed02: a0,b0,c0 / seed12: a1,b1 (ReLU)      */
    PUR_MUL_TRIPLE = 6, /* seed02: a0,b0,c0 / seed12: a1,b1 (product)   */
    PUR_ABY3 = 7,       /* seed02: [r]_0, [r']_0 / seed12: [r]_1         */
    PUR_RSS_T = 8,      /* seed012: alpha_0..2 (sharing of t)            */
    PUR_RSS_S = 9,      /* seed2: s / seed012: [s]_1 / seed12: [s]_2     */
    PUR_RSS_Z = 10,     /* seed012: gamma_0..2, zero sharing of [s][t]   */
    PUR_RSS_ZR = 11,    /* seed012: zero sharing of the RSS ReLU product */
    PUR_B1_MASK = 12    /* seed01: r_k, z_k of slot k, Bicoptor 1.0-style */
};

uint32_t orc_stream_word(uint64_t seed, int pair, int purpose, uint32_t tensor_id,
                         uint64_t elem, uint64_t j)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)elem, tensor_id, (uint32_t)(j / 4),
                       ((uint32_t)pair << 24) | ((uint32_t)purpose << 16) |
                           (uint32_t)((elem >> 32) & 0xffffu)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[j % 4];
}

/* Ring element number j of a stream: one word for l <= 32, two words (low
 * word first) for l > 32, reduced mod 2^l. */
static uint64_t stream_ring(uint64_t seed, int pair, int purpose, uint32_t tid,
                            uint64_t elem, uint64_t j, int ell)
{
    if (ell <= 32)
        return rmod(orc_stream_word(seed, pair, purpose, tid, elem, j), ell);
    uint64_t lo = orc_stream_word(seed, pair, purpose, tid, elem, 2 * j);
    uint64_t hi = orc_stream_word(seed, pair, purpose, tid, elem, 2 * j + 1);
    return rmod(lo | (hi << 32), ell);
}

/* ------------------------------------------------------------------------- */
/* Prime for the modulo switch.                                              */
/* READING: "log2 p = l'+1" (Sec. 5.3, Table notation) with the correctness  */
/* argument needing p > 2^l'; the oracle takes the smallest prime above      */
/* 2^lx, found by trial division.                                            */
/* ------------------------------------------------------------------------- */

static int is_prime_u64(uint64_t q)
{
    if (q < 2) return 0;
    for (uint64_t d = 2; d * d <= q; d++)
        if (q % d == 0) return 0;
    return 1;
}

uint32_t orc_prime_above(int lx)
{
    uint64_t q = ((uint64_t)1 << lx) + 1;
    while (!is_prime_u64(q)) q++;
    return (uint32_t)q;
}

/* ------------------------------------------------------------------------- */
/* Fixed-point encoding (Sec. 2.2): x -> round(x * 2^f) mod 2^l, with        */
/* l_x = l_x^int + l_x^frac.  READING: round half to even (the paper does    */
/* not say); nearbyint() in the default rounding mode does exactly that.     */
/* ------------------------------------------------------------------------- */

void orc_encode(const double *x, size_t n, int f, int ell, uint64_t *out)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        double scaled = nearbyint(ldexp(x[i], f));
        int64_t v = (int64_t)scaled;
        out[i] = rmod((uint64_t)v, ell);
    }
}

/* Signed value of a ring element: x in [0, 2^(l-1)) is positive. */
void orc_to_signed(const uint64_t *v, size_t n, int ell, int64_t *out)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint64_t a = rmod(v[i], ell);
        if (ell < 64 && (a >> (ell - 1)))
            out[i] = (int64_t)a - (int64_t)((uint64_t)1 << ell);
        else
            out[i] = (int64_t)a;
    }
}

/* ------------------------------------------------------------------------- */
/* 2-of-2 additive sharing (Sec. 2.2): [x]_0 = x + R, [x]_1 = -R (mod 2^l).  */
/* ------------------------------------------------------------------------- */

void orc_share_with_r(int ell, uint64_t x, uint64_t r, uint64_t *s0, uint64_t *s1)
{
    *s0 = rmod(x + r, ell);
    *s1 = rneg(r, ell);
}

static uint64_t elem_index(const uint64_t *idx, size_t i) { return idx ? idx[i] : (uint64_t)i; }

void orc_share(int ell, const uint64_t *x, const uint64_t *idx, size_t n, uint64_t seed,
               uint32_t tid, uint64_t *s0, uint64_t *s1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint64_t R = stream_ring(seed, PAIR_DEALER, PUR_SHARE, tid, elem_index(idx, i), 0, ell);
        orc_share_with_r(ell, x[i], R, &s0[i], &s1[i]);
    }
}

void orc_reconstruct(int ell, const uint64_t *s0, const uint64_t *s1, size_t n, uint64_t *x)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) x[i] = rmod(s0[i] + s1[i], ell);
}

/* ------------------------------------------------------------------------- */
/* Alg. smltrc (SecureML probabilistic truncation), per party.               */
/*   P0: cut([x]_0, k) mod 2^l;  P1: 2^l - cut(2^l - [x]_1, k) mod 2^l.      */
/* READING: 2^l - [x]_1 is reduced mod 2^l before the cut (so [x]_1 = 0      */
/* gives 0).                                                                  */
/* ------------------------------------------------------------------------- */

static uint64_t smltrc_p0(uint64_t s0, int ell, int k) { return rmod(orc_cut(s0, ell, k, 0), ell); }
static uint64_t smltrc_p1(uint64_t s1, int ell, int k)
{
    uint64_t a = rneg(s1, ell);                 /* 2^l - [x]_1 mod 2^l */
    return rneg(orc_cut(a, ell, k, 0), ell);    /* 2^l - cut(., k) mod 2^l */
}

void orc_trunc_prob(int ell, int k, const uint64_t *s0, const uint64_t *s1, size_t n,
                    uint64_t *o0, uint64_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        o0[i] = smltrc_p0(s0[i], ell, k);
        o1[i] = smltrc_p1(s1[i], ell, k);
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. newtrc2 (deterministic truncation keeping bits k1 .. l-k2-1), per    */
/* party, outputs in Z_{2^(l-k1-k2)}.  Alg. newtrc is the case k2 = 0.       */
/* READING: k1 counts the low bits dropped and k2 the high bits dropped; the */
/* worked example of Sec. 5.1 (k1 = 4, k2 = 1 -> 100) fixes this order.      */
/* ------------------------------------------------------------------------- */

static uint64_t newtrc_p0(uint64_t s0, int ell, int k1, int k2)
{
    return rmod(orc_cut(s0, ell, k1, k2), ell - k1 - k2);
}
static uint64_t newtrc_p1(uint64_t s1, int ell, int k1, int k2)
{
    uint64_t a = rneg(s1, ell);                          /* 2^l - [x]_1 mod 2^l */
    return rneg(orc_cut(a, ell, k1, k2), ell - k1 - k2); /* 2^l - cut(.) mod 2^(l-k1-k2) */
}

void orc_trunc_det(int ell, int k1, int k2, const uint64_t *s0, const uint64_t *s1, size_t n,
                   uint64_t *o0, uint64_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        o0[i] = newtrc_p0(s0[i], ell, k1, k2);
        o1[i] = newtrc_p1(s1[i], ell, k1, k2);
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. modswitch: shares in Z_{2^l'} -> shares in Z_p with zero <-> zero.   */
/*   P0: 2^l' mod p if [x]_0 = 0, else [x]_0 mod p;                          */
/*   P1: p + [x]_1 - 2^l' mod p.                                             */
/* ------------------------------------------------------------------------- */

static uint32_t modswitch_p0(uint64_t a, int lp, uint32_t p)
{
    uint64_t pow2 = (uint64_t)1 << lp;
    if (a == 0) return (uint32_t)(pow2 % p);
    return (uint32_t)(a % p);
}
static uint32_t modswitch_p1(uint64_t b, int lp, uint32_t p)
{
    uint64_t pow2 = (uint64_t)1 << lp;
    /* p + b - 2^l' is in (p - 2^l', p + 2^l'), never negative since b >= 0
       and p > 2^l'. */
    return (uint32_t)(((uint64_t)p + b - pow2) % p);
}

void orc_mod_switch(int lp, uint32_t p, const uint64_t *s0, const uint64_t *s1, size_t n,
                    uint32_t *o0, uint32_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        o0[i] = modswitch_p0(rmod(s0[i], lp), lp, p);
        o1[i] = modswitch_p1(rmod(s1[i], lp), lp, p);
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. aby3trc (ABY3 probabilistic truncation) between P0 and P1, with P2  */
/* dealing the pair (r, r' = r / 2^k): [r]_0 and [r']_0 from seed02, [r]_1  */
/* from seed12; P2 sends [r']_1 = r' - [r']_0 to P1 (preprocessing).         */
/* Online both open alpha = x + r; P0 sets alpha / 2^k - [r']_0 and P1 sets  */
/* -[r']_1 (the public alpha / 2^k is added by P0 alone).                    */
/* READING: / 2^k is floor division of the two's-complement (signed) value. */
/* Sec. 4.1's claim that a fixed r = 2^26 never triggers e1 for 62-bit      */
/* inputs holds for negative inputs only under this reading.                 */
/* ------------------------------------------------------------------------- */

static uint64_t floor_div_pow2_signed(uint64_t a, int ell, int k)
{
    __int128 v = (__int128)rmod(a, ell);
    if (ell < 128 && (v >> (ell - 1)) & 1) v -= ((__int128)1 << ell);   /* signed value */
    __int128 d = (__int128)1 << k;
    __int128 q = v >= 0 ? v / d : -((-v + d - 1) / d);                  /* floor */
    return rmod((uint64_t)q, ell);
}

/* One element of Alg. aby3trc with the preprocessing randomness passed in:
 * r0 = [r]_0, r1 = [r]_1 (r = r0 + r1), rp0 = [r']_0.  Returns the shares. */
void orc_aby3_core(int ell, int k, uint64_t s0, uint64_t s1, uint64_t r0, uint64_t r1,
                   uint64_t rp0, uint64_t *o0, uint64_t *o1)
{
    uint64_t r = rmod(r0 + r1, ell);                       /* known to P2 */
    uint64_t rp = floor_div_pow2_signed(r, ell, k);        /* r' = r / 2^k */
    uint64_t rp1 = rmod(rp - rp0, ell);                    /* P2 -> P1 */
    uint64_t alpha = rmod((s0 + r0) + (s1 + r1), ell);     /* opened */
    *o0 = rmod(floor_div_pow2_signed(alpha, ell, k) - rp0, ell);
    *o1 = rneg(rp1, ell);
}

/* fixed_r != 0 reproduces the implementation shortcut of Sec. 4.1: r is
 * the constant fixed_r (its shares stay random: [r]_1 = fixed_r - [r]_0). */
void orc_trunc_aby3(int ell, int k, const uint64_t *s0, const uint64_t *s1, const uint64_t *idx,
                    size_t n, uint64_t seed, uint32_t tid, uint64_t fixed_r, uint64_t *o0,
                    uint64_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint64_t elem = elem_index(idx, i);
        uint64_t r0 = stream_ring(seed, PAIR_02, PUR_ABY3, tid, elem, 0, ell);
        uint64_t rp0 = stream_ring(seed, PAIR_02, PUR_ABY3, tid, elem, 1, ell);
        uint64_t r1 = stream_ring(seed, PAIR_12, PUR_ABY3, tid, elem, 0, ell);
        if (fixed_r) r1 = rmod(fixed_r - r0, ell);
        orc_aby3_core(ell, k, s0[i], s1[i], r0, r1, rp0, &o0[i], &o1[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Beaver multiplication (Table notation, Sec. 2.3; Alg. relu pre-          */
/* processing): the triple comes from the pre-shared seeds, P2 completes     */
/* [c]_1 = (a0 + a1)(b0 + b1) - [c]_0 and sends it to P1.  d = x - a and     */
/* e = y - b are opened; [xy] = de + d[b] + e[a] + [c], de added by P0.      */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t a0, b0, c0, a1, b1, c1; } triple_t;

static triple_t draw_triple(uint64_t seed, int purpose, uint32_t tid, uint64_t elem, int ell)
{
    triple_t T;
    T.a0 = stream_ring(seed, PAIR_02, purpose, tid, elem, 0, ell);
    T.b0 = stream_ring(seed, PAIR_02, purpose, tid, elem, 1, ell);
    T.c0 = stream_ring(seed, PAIR_02, purpose, tid, elem, 2, ell);
    T.a1 = stream_ring(seed, PAIR_12, purpose, tid, elem, 0, ell);
    T.b1 = stream_ring(seed, PAIR_12, purpose, tid, elem, 1, ell);
    /* P2 knows both halves and completes the triple. */
    T.c1 = rmod((T.a0 + T.a1) * (T.b0 + T.b1) - T.c0, ell);
    return T;
}

void orc_mul_beaver(int ell, const uint64_t *x0, const uint64_t *x1, const uint64_t *y0,
                    const uint64_t *y1, const uint64_t *idx, size_t n, uint64_t seed,
                    uint32_t tid, uint64_t *o0, uint64_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        triple_t T = draw_triple(seed, PUR_MUL_TRIPLE, tid, elem_index(idx, i), ell);
        /* openings: each party sends its share of x - a and of y - b */
        uint64_t d = rmod((x0[i] - T.a0) + (x1[i] - T.a1), ell);
        uint64_t e = rmod((y0[i] - T.b0) + (y1[i] - T.b1), ell);
        o0[i] = rmod(d * e + d * T.b0 + e * T.a0 + T.c0, ell);
        o1[i] = rmod(d * T.b1 + e * T.a1 + T.c1, ell);
    }
}

/* Alg. linear (truncate-then-multiply): P_i truncates its shares of x by
 * kx bits and of y by ky bits with Alg. smltrc (kx + ky = l_x^frac; for an
 * odd precision one input loses one bit more), then the Beaver product of
 * the truncated shares gives shares of trc(x y, l_x^frac). */
void orc_trunc_then_mul(int ell, int kx, int ky, const uint64_t *x0, const uint64_t *x1,
                        const uint64_t *y0, const uint64_t *y1, const uint64_t *idx, size_t n,
                        uint64_t seed, uint32_t tid, uint64_t *o0, uint64_t *o1)
{
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint64_t tx0 = smltrc_p0(x0[i], ell, kx), tx1 = smltrc_p1(x1[i], ell, kx);
        uint64_t ty0 = smltrc_p0(y0[i], ell, ky), ty1 = smltrc_p1(y1[i], ell, ky);
        uint64_t e = elem_index(idx, i);
        orc_mul_beaver(ell, &tx0, &tx1, &ty0, &ty1, &e, 1, seed, tid, &o0[i], &o1[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. drelu (UBL Bicoptor 2.0 DReLU), steps 1-9, for one element, with     */
/* the randomness that P0 and P1 draw from seed01 passed in:                 */
/*   t          flip bit (step 1)                                            */
/*   fy[1..lx]  32-bit words for the shuffle (step 6)                        */
/*   r[k],z[k]  mask in Z_p^* and reshare value in Z_p of message slot k     */
/* Writes P0's and P1's messages to P2 and P2's bit DReLU'.                  */
/* ------------------------------------------------------------------------- */

typedef struct { int ell, lx, c; uint32_t p; } orc_params;

#define MAXL 64

int orc_drelu_core(const orc_params *P, uint64_t s0, uint64_t s1, int t, const uint32_t *fy,
                   const uint32_t *r, const uint32_t *z, uint32_t *msg0, uint32_t *msg1)
{
    const int ell = P->ell, lx = P->lx, c = P->c;
    const uint32_t p = P->p;
    const int L = lx + 1;
    uint64_t u0[MAXL], u1[MAXL], v0[MAXL], v1[MAXL];
    uint32_t m0[MAXL], m1[MAXL], sh0[MAXL], sh1[MAXL], w[MAXL];
    int perm[MAXL];

    /* Steps 1-2: both parties flip their share by (-1)^t. */
    if (t) { s0 = rneg(s0, ell); s1 = rneg(s1, ell); }

    /* Step 3: [u_i] = [trc(x, i, l - lx - i)] mod 2^lx for i in [0, lx], with
       the window moved up by the key-bit offset c (Sec. 6.1):
       k1 = c + i, k2 = l - lx - c - i. */
    for (int i = 0; i <= lx; i++) {
        int k1 = c + i, k2 = ell - lx - c - i;
        u0[i] = newtrc_p0(s0, ell, k1, k2);
        u1[i] = newtrc_p1(s1, ell, k1, k2);
    }

    /* Step 4: [v_i] = [u_i] + [u_(i+1)] - 1, [v_lx] = [u_lx] - 1 (mod 2^lx).
       READING: the public constant -1 is applied by P0 alone. */
    for (int i = 0; i < lx; i++) {
        v0[i] = rmod(u0[i] + u0[i + 1] - 1, lx);
        v1[i] = rmod(u1[i] + u1[i + 1], lx);
    }
    v0[lx] = rmod(u0[lx] - 1, lx);
    v1[lx] = rmod(u1[lx], lx);

    /* Step 5: Alg. modswitch, Z_{2^lx} -> Z_p. */
    for (int i = 0; i <= lx; i++) {
        m0[i] = modswitch_p0(v0[i], lx, p);
        m1[i] = modswitch_p1(v1[i], lx, p);
    }

    /* Step 6: shuffle with seed01.  READING: a Fisher-Yates shuffle of the
       slots 0..lx starting from the identity; for j = lx down to 1 the swap
       partner is floor(W * (j+1) / 2^32) with W = fy[lx - j + 1].  Message
       slot k carries the value at perm[k]. */
    for (int k = 0; k < L; k++) perm[k] = k;
    for (int j = lx; j >= 1; j--) {
        uint32_t W = fy[lx - j + 1];
        int partner = (int)(((uint64_t)W * (uint64_t)(j + 1)) >> 32);
        int tmp = perm[j]; perm[j] = perm[partner]; perm[partner] = tmp;
    }
    for (int k = 0; k < L; k++) { sh0[k] = m0[perm[k]]; sh1[k] = m1[perm[k]]; }

    /* Step 7: mask with r_k in Z_p^*, w_k = v_k * r_k mod p. */
    for (int k = 0; k < L; k++) {
        sh0[k] = (uint32_t)(((uint64_t)sh0[k] * r[k]) % p);
        sh1[k] = (uint32_t)(((uint64_t)sh1[k] * r[k]) % p);
    }

    /* Step 8: reshare with z_k (READING: P0 adds, P1 subtracts) and send. */
    for (int k = 0; k < L; k++) {
        msg0[k] = (uint32_t)(((uint64_t)sh0[k] + z[k]) % p);
        msg1[k] = (uint32_t)(((uint64_t)sh1[k] + p - z[k]) % p);
    }

    /* Step 9: P2 reconstructs every w_k and sets DReLU' = 1 if one is 0. */
    int dprime = 0;
    for (int k = 0; k < L; k++) {
        w[k] = (uint32_t)(((uint64_t)msg0[k] + msg1[k]) % p);
        if (w[k] == 0) dprime = 1;
    }
    return dprime;
}

/* 2^-32 mod p, by Fermat's little theorem: (2^32)^(p-2) mod p. */
static uint32_t inv_two32_mod_p(uint32_t p)
{
    uint64_t base = ((uint64_t)1 << 32) % p, acc = 1, e = (uint64_t)p - 2;
    while (e) {
        if (e & 1) acc = (acc * base) % p;
        base = (base * base) % p;
        e >>= 1;
    }
    return (uint32_t)acc;
}

/* The seed01 draws of one element: t, the shuffle words, and (r_k, z_k).
 * READING: from two 64-bit words W, W' of the slot's mask block (words
 * 4k..4k+3, low word first), rho_k = 1 + floor(W (p-1) / 2^64) and
 * z_k = floor(W' p / 2^64), each within 2^-(64 - log2 p) of uniform; the
 * mask is r_k = rho_k * 2^-32 mod p, which is as uniform on Z_p^* as rho_k
 * (multiplying by the unit 2^-32 permutes Z_p^*). */
static void draw_seed01(const orc_params *P, uint64_t seed, uint32_t tid, uint64_t elem,
                        uint32_t inv32, int *t, uint32_t *fy, uint32_t *r, uint32_t *z)
{
    const int L = P->lx + 1;
    *t = (int)(orc_stream_word(seed, PAIR_01, PUR_PERM, tid, elem, 0) & 1u);
    for (int j = 1; j < L; j++) fy[j] = orc_stream_word(seed, PAIR_01, PUR_PERM, tid, elem, j);
    for (int k = 0; k < L; k++) {
        uint64_t wr = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k) |
                      ((uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k + 1) << 32);
        uint64_t wz = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k + 2) |
                      ((uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k + 3) << 32);
        uint32_t rho = 1u + (uint32_t)(((u128)wr * (u128)(P->p - 1u)) >> 64);
        r[k] = (uint32_t)(((uint64_t)rho * inv32) % P->p);
        z[k] = (uint32_t)(((u128)wz * (u128)P->p) >> 64);
    }
}

/* Parameter checks shared by DReLU and ReLU: the window needs c + 2 lx <= l
 * (k2 >= 0 at i = lx), p must lie in (2^lx, 2^(lx+1)). */
static int check_params(const orc_params *P)
{
    if (P->ell < 2 || P->ell > 64) return -1;
    if (P->lx < 1 || P->lx > 31 || P->lx + 1 > MAXL) return -1;
    if (P->c < 0 || P->c + 2 * P->lx > P->ell) return -1;
    if ((uint64_t)P->p <= ((uint64_t)1 << P->lx) || (uint64_t)P->p >= ((uint64_t)1 << (P->lx + 1)))
        return -1;
    if (!is_prime_u64(P->p)) return -1;
    return 0;
}

/* Audit view of one call: what each party sent (NULL = not wanted). */
typedef struct {
    uint32_t *w0;        /* P0 -> P2, n * (lx+1) values in Z_p              */
    uint32_t *w1;        /* P1 -> P2, n * (lx+1) values in Z_p              */
    uint64_t *reply;     /* P2 -> P1: [DReLU']_1 (DReLU); P2 -> P0,P1: e (ReLU) */
    uint64_t *open0;     /* P0 -> P1: [x]_0 - [a]_0 (ReLU)                  */
    uint64_t *open1;     /* P1 -> P0: [x]_1 - [a]_1 (ReLU)                  */
    uint64_t *pre_c1;    /* P2 -> P1 preprocessing: [c]_1 (ReLU)             */
    uint8_t *t;          /* the flip bit (seed01)                           */
    uint8_t *dprime;     /* P2's DReLU'                                     */
} orc_audit;

/* Steps 10-11 of Alg. drelu: P2 returns DReLU' as shares in Z_{2^l};
 * READING: [DReLU']_0 = d0 is drawn from seed02 by P0 and P2 alike, so only
 * [DReLU']_1 = DReLU' - d0 travels (to P1).  Unflip:
 * [DReLU]_0 = t + (1-2t)[DReLU']_0, [DReLU]_1 = (1-2t)[DReLU']_1; the public
 * t is added by P0 alone. */
int orc_drelu(const orc_params *P, const uint64_t *s0, const uint64_t *s1, const uint64_t *idx,
              size_t n, uint64_t seed, uint32_t tid, uint64_t *o0, uint64_t *o1,
              const orc_audit *audit, int threads)
{
    if (check_params(P)) return -1;
    const int ell = P->ell, L = P->lx + 1;
    const uint32_t inv32 = inv_two32_mod_p(P->p);
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long ii = 0; ii < (long long)n; ii++) {
        size_t i = (size_t)ii;
        uint64_t elem = elem_index(idx, i);
        int t;
        uint32_t fy[MAXL], r[MAXL], z[MAXL], msg0[MAXL], msg1[MAXL];
        draw_seed01(P, seed, tid, elem, inv32, &t, fy, r, z);
        int dprime = orc_drelu_core(P, s0[i], s1[i], t, fy, r, z, msg0, msg1);
        uint64_t d0 = stream_ring(seed, PAIR_02, PUR_REPLY, tid, elem, 0, ell);
        uint64_t d1 = rmod((uint64_t)dprime - d0, ell);
        uint64_t one_m2t = rmod((uint64_t)1 - 2 * (uint64_t)t, ell);
        o0[i] = rmod((uint64_t)t + one_m2t * d0, ell);
        o1[i] = rmod(one_m2t * d1, ell);
        if (audit) {
            if (audit->w0) memcpy(audit->w0 + i * L, msg0, sizeof(uint32_t) * L);
            if (audit->w1) memcpy(audit->w1 + i * L, msg1, sizeof(uint32_t) * L);
            if (audit->reply) audit->reply[i] = d1;
            if (audit->t) audit->t[i] = (uint8_t)t;
            if (audit->dprime) audit->dprime[i] = (uint8_t)dprime;
        }
    }
    return 0;
}

/* Alg. relu (UBL Bicoptor 2.0 ReLU).  P2 answers e = DReLU' - b instead of
 * shares of DReLU'; P0 and P1 open d = x - a and finish
 * [ReLU] = t[x] + (1-2t)(de + d[b] + e[a] + [c]), de added by P0 alone.
 * READING: x here is the input before the flip of step 2. */
int orc_relu(const orc_params *P, const uint64_t *s0, const uint64_t *s1, const uint64_t *idx,
             size_t n, uint64_t seed, uint32_t tid, uint64_t *o0, uint64_t *o1,
             const orc_audit *audit, int threads)
{
    if (check_params(P)) return -1;
    const int ell = P->ell, L = P->lx + 1;
    const uint32_t inv32 = inv_two32_mod_p(P->p);
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long ii = 0; ii < (long long)n; ii++) {
        size_t i = (size_t)ii;
        uint64_t elem = elem_index(idx, i);
        /* preprocessing: the triple */
        triple_t T = draw_triple(seed, PUR_RELU_TRIPLE, tid, elem, ell);
        /* P0, P1 run Alg. drelu up to step 8; P2 runs step 9 */
        int t;
        uint32_t fy[MAXL], r[MAXL], z[MAXL], msg0[MAXL], msg1[MAXL];
        draw_seed01(P, seed, tid, elem, inv32, &t, fy, r, z);
        int dprime = orc_drelu_core(P, s0[i], s1[i], t, fy, r, z, msg0, msg1);
        /* P2 responds e = DReLU' - b */
        uint64_t e = rmod((uint64_t)dprime - (T.b0 + T.b1), ell);
        /* P0 and P1 open d = x - a */
        uint64_t open0 = rmod(s0[i] - T.a0, ell), open1 = rmod(s1[i] - T.a1, ell);
        uint64_t d = rmod(open0 + open1, ell);
        uint64_t xd0 = rmod(d * e + d * T.b0 + e * T.a0 + T.c0, ell);
        uint64_t xd1 = rmod(d * T.b1 + e * T.a1 + T.c1, ell);
        uint64_t one_m2t = rmod((uint64_t)1 - 2 * (uint64_t)t, ell);
        o0[i] = rmod((uint64_t)t * s0[i] + one_m2t * xd0, ell);
        o1[i] = rmod((uint64_t)t * s1[i] + one_m2t * xd1, ell);
        if (audit) {
            if (audit->w0) memcpy(audit->w0 + i * L, msg0, sizeof(uint32_t) * L);
            if (audit->w1) memcpy(audit->w1 + i * L, msg1, sizeof(uint32_t) * L);
            if (audit->reply) audit->reply[i] = e;
            if (audit->open0) audit->open0[i] = open0;
            if (audit->open1) audit->open1[i] = open1;
            if (audit->pre_c1) audit->pre_c1[i] = T.c1;
            if (audit->t) audit->t[i] = (uint8_t)t;
            if (audit->dprime) audit->dprime[i] = (uint8_t)dprime;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Alg. drelu2 (RSS Bicoptor 2.0 DReLU) and the RSS ReLU.  2-of-3 replicated */
/* sharing: x = x0 + x1 + x2, P0 holds (x0, x1), P1 (x1, x2), P2 (x2, x0);  */
/* component arrays x0, x1, x2 in and y0, y1, y2 out.                         */
/* Preprocessing: t from seed01; alpha_i from seed012, beta_i = alpha_i -   */
/* alpha_(i-1), [t] = (beta_0, beta_1 + t, beta_2); s a bit from seed2,      */
/* [s]_1 from seed012, [s]_2 from seed12, [s]_0 = s - [s]_1 - [s]_2 (P2 ->   */
/* P0); [s xor t] = [s] + [t] - 2 [s][t].                                     */
/* READING: [s][t] is the replicated product (each P_i forms                  */
/* s_i t_i + s_i t_(i+1) + s_(i+1) t_i plus a zero sharing                    */
/* gamma_i - gamma_(i+1) and sends it to P_(i-1)); the paper names the       */
/* product but not its protocol.                                              */
/* Online: P0 runs Alg. drelu on [x]_0 + [x]_1, P1 on [x]_2 (steps 1-8 with  */
/* the same seed01 draws); P2 gets DReLU', sends d'' = s xor DReLU' to P0    */
/* and P1; all set [DReLU] = d'' + [s xor t] - 2 d'' [s xor t] (the public  */
/* d'' added to component 0).  RSS ReLU: the replicated product              */
/* [x] [DReLU] with its own zero sharing (Sec. "How to construct the RSS     */
/* ... protocols").                                                          */
/* ------------------------------------------------------------------------- */

static void rss_mul(int ell, const uint64_t a[3], const uint64_t b[3], const uint64_t g[3],
                    uint64_t out[3])
{
    for (int i = 0; i < 3; i++) {
        int j = (i + 1) % 3;
        out[i] = rmod(a[i] * b[i] + a[i] * b[j] + a[j] * b[i] + g[i] - g[j], ell);
    }
}

int orc_rss_drelu(const orc_params *P, const uint64_t *x0, const uint64_t *x1, const uint64_t *x2,
                  const uint64_t *idx, size_t n, uint64_t seed, uint32_t tid, int relu,
                  uint64_t *y0, uint64_t *y1, uint64_t *y2, uint8_t *dprime_out, int threads)
{
    if (check_params(P)) return -1;
    const int ell = P->ell;
    const uint32_t inv32 = inv_two32_mod_p(P->p);
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long ii = 0; ii < (long long)n; ii++) {
        size_t i = (size_t)ii;
        uint64_t elem = elem_index(idx, i);
        int t;
        uint32_t fy[MAXL], r[MAXL], z[MAXL], msg0[MAXL], msg1[MAXL];
        draw_seed01(P, seed, tid, elem, inv32, &t, fy, r, z);
        /* preprocessing: [t], [s], [s xor t] */
        uint64_t al[3], T[3], S[3], g[3], ST[3], X[3];
        for (int j = 0; j < 3; j++) al[j] = stream_ring(seed, PAIR_012, PUR_RSS_T, tid, elem, j, ell);
        T[0] = rmod(al[0] - al[2], ell);
        T[1] = rmod(al[1] - al[0] + (uint64_t)t, ell);
        T[2] = rmod(al[2] - al[1], ell);
        uint64_t sbit = orc_stream_word(seed, PAIR_2, PUR_RSS_S, tid, elem, 0) & 1u;
        S[1] = stream_ring(seed, PAIR_012, PUR_RSS_S, tid, elem, 0, ell);
        S[2] = stream_ring(seed, PAIR_12, PUR_RSS_S, tid, elem, 0, ell);
        S[0] = rmod(sbit - S[1] - S[2], ell);
        for (int j = 0; j < 3; j++) g[j] = stream_ring(seed, PAIR_012, PUR_RSS_Z, tid, elem, j, ell);
        rss_mul(ell, S, T, g, ST);
        for (int j = 0; j < 3; j++) X[j] = rmod(S[j] + T[j] - 2 * ST[j], ell);
        /* online: Alg. drelu between P0 ([x]_0 + [x]_1) and P1 ([x]_2) */
        int dprime = orc_drelu_core(P, rmod(x0[i] + x1[i], ell), x2[i], t, fy, r, z, msg0, msg1);
        uint64_t dd = (sbit ^ (uint64_t)dprime);            /* d'' = s xor DReLU' */
        uint64_t Y[3];
        for (int j = 0; j < 3; j++) Y[j] = rmod(X[j] - 2 * dd * X[j] + (j == 0 ? dd : 0), ell);
        if (relu) {
            uint64_t xr[3] = {x0[i], x1[i], x2[i]}, gr[3], Z[3];
            for (int j = 0; j < 3; j++)
                gr[j] = stream_ring(seed, PAIR_012, PUR_RSS_ZR, tid, elem, j, ell);
            rss_mul(ell, xr, Y, gr, Z);
            for (int j = 0; j < 3; j++) Y[j] = Z[j];
        }
        y0[i] = Y[0]; y1[i] = Y[1]; y2[i] = Y[2];
        if (dprime_out) dprime_out[i] = (uint8_t)dprime;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The Bicoptor 1.0-style DReLU that this paper improves on, as it describes */
/* it by contrast (Table "compare"; Sec. "sub:cmp"; the notes on steps 3 and */
/* 4 of Alg. drelu):                                                          */
/*   step 3  SecureML truncations (Alg. smltrc) in Z_{2^l}, not Z_{2^lx}, at  */
/*           every key-bit position c + i, i = 0..lx                          */
/*   step 4  recursive sums S_i = sum_{k=i..lx} u_k, v_i = S_i - 1 (P0 holds  */
/*           the constant), instead of adjacent pairs                         */
/*   no modulo switch: masking, shuffling, resharing and P2's zero test stay  */
/*   in Z_{2^l}; each party sends lx+1 ring elements, (lx+1) l bits          */
/*   no u* term (DReLU(0) is t, as in Bicoptor 2.0)                           */
/* READING: the mask r_k must keep zero <=> zero in Z_{2^l}, so it is a       */
/* random odd element (a unit); r_k = (W | 1) mod 2^l and z_k = W' mod 2^l   */
/* from the two 64-bit words of slot k's seed01 block (purpose PUR_B1_MASK). */
/* The shuffle, t, the reply and the ReLU triple are drawn as in Bicoptor    */
/* 2.0.  The paper's table counts l_x l bits per party; its text (2,048 and  */
/* 512 bits at l_x = 31 and 7) counts the l_x + 1 values sent here.           */
/* ------------------------------------------------------------------------- */

/* Steps 1-9 for one element with the randomness passed in (r[k] odd). */
int orc_drelu_b1_core(const orc_params *P, uint64_t s0, uint64_t s1, int t, const uint32_t *fy,
                      const uint64_t *r, const uint64_t *z, uint64_t *msg0, uint64_t *msg1)
{
    const int ell = P->ell, lx = P->lx, c = P->c;
    const int L = lx + 1;
    uint64_t u0[MAXL], u1[MAXL], v0[MAXL], v1[MAXL], sh0[MAXL], sh1[MAXL];
    int perm[MAXL];

    /* Steps 1-2: flip by (-1)^t. */
    if (t != 0) { s0 = rneg(s0, ell); s1 = rneg(s1, ell); }

    /* Step 3: Alg. smltrc of each party's share by c + i bits, in Z_{2^l}. */
    for (int i = 0; i <= lx; i++) {
        u0[i] = smltrc_p0(s0, ell, c + i);
        u1[i] = smltrc_p1(s1, ell, c + i);
    }

    /* Step 4: recursive sums from the top, minus one (P0). */
    uint64_t acc0 = 0, acc1 = 0;
    for (int i = lx; i >= 0; i--) {
        acc0 = rmod(acc0 + u0[i], ell);
        acc1 = rmod(acc1 + u1[i], ell);
        v0[i] = rmod(acc0 - 1, ell);
        v1[i] = acc1;
    }

    /* Step 6: the shuffle of Bicoptor 2.0 (Fisher-Yates from the identity). */
    for (int k = 0; k < L; k++) perm[k] = k;
    for (int j = lx; j >= 1; j--) {
        uint64_t word = fy[lx - j + 1];
        int q = (int)((word * (uint64_t)(j + 1)) >> 32);
        int tmp = perm[j]; perm[j] = perm[q]; perm[q] = tmp;
    }
    for (int k = 0; k < L; k++) { sh0[k] = v0[perm[k]]; sh1[k] = v1[perm[k]]; }

    /* Steps 7-8: mask by the unit r_k, reshare with z_k (P0 adds, P1
       subtracts), all in Z_{2^l}. */
    for (int k = 0; k < L; k++) {
        msg0[k] = rmod(sh0[k] * r[k] + z[k], ell);
        msg1[k] = rmod(sh1[k] * r[k] - z[k], ell);
    }

    /* Step 9: P2 reconstructs every w_k in Z_{2^l}; DReLU' = 1 if one is 0. */
    int dprime = 0;
    for (int k = 0; k < L; k++)
        if (rmod(msg0[k] + msg1[k], ell) == 0) dprime = 1;
    return dprime;
}

static void draw_b1(const orc_params *P, uint64_t seed, uint32_t tid, uint64_t elem, int *t,
                    uint32_t *fy, uint64_t *r, uint64_t *z)
{
    const int L = P->lx + 1;
    *t = (int)(orc_stream_word(seed, PAIR_01, PUR_PERM, tid, elem, 0) & 1u);
    for (int j = 1; j < L; j++) fy[j] = orc_stream_word(seed, PAIR_01, PUR_PERM, tid, elem, j);
    for (int k = 0; k < L; k++) {
        uint64_t wr = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_B1_MASK, tid, elem, 4 * k) |
                      ((uint64_t)orc_stream_word(seed, PAIR_01, PUR_B1_MASK, tid, elem, 4 * k + 1) << 32);
        uint64_t wz = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_B1_MASK, tid, elem, 4 * k + 2) |
                      ((uint64_t)orc_stream_word(seed, PAIR_01, PUR_B1_MASK, tid, elem, 4 * k + 3) << 32);
        r[k] = rmod(wr | 1u, P->ell);
        z[k] = rmod(wz, P->ell);
    }
}

/* The parameters of the 1.0-style protocol: no prime (p is ignored). */
static int check_params_b1(const orc_params *P)
{
    if (P->ell < 2 || P->ell > 64) return -1;
    if (P->lx < 1 || P->lx > 31 || P->lx + 1 > MAXL) return -1;
    if (P->c < 0 || P->c + P->lx >= P->ell) return -1;
    return 0;
}

/* DReLU (relu = 0) or ReLU (relu = 1) of the 1.0-style protocol; steps 10-11
   and Alg. relu's Beaver finish exactly as in Bicoptor 2.0.  msgs (optional):
   w0 then w1, each n * (lx+1) ring elements, slot-major per element. */
int orc_b1(const orc_params *P, int relu, const uint64_t *s0, const uint64_t *s1,
           const uint64_t *idx, size_t n, uint64_t seed, uint32_t tid, uint64_t *o0,
           uint64_t *o1, uint64_t *w0, uint64_t *w1, uint8_t *dprime_out, int threads)
{
    if (check_params_b1(P)) return -1;
    const int ell = P->ell, L = P->lx + 1;
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (long long ii = 0; ii < (long long)n; ii++) {
        size_t i = (size_t)ii;
        uint64_t elem = elem_index(idx, i);
        int t;
        uint32_t fy[MAXL];
        uint64_t r[MAXL], z[MAXL], msg0[MAXL], msg1[MAXL];
        draw_b1(P, seed, tid, elem, &t, fy, r, z);
        int dprime = orc_drelu_b1_core(P, s0[i], s1[i], t, fy, r, z, msg0, msg1);
        uint64_t one_m2t = rmod((uint64_t)1 - 2 * (uint64_t)t, ell);
        if (!relu) {
            uint64_t d0 = stream_ring(seed, PAIR_02, PUR_REPLY, tid, elem, 0, ell);
            uint64_t d1 = rmod((uint64_t)dprime - d0, ell);
            o0[i] = rmod((uint64_t)t + one_m2t * d0, ell);
            o1[i] = rmod(one_m2t * d1, ell);
        } else {
            triple_t T = draw_triple(seed, PUR_RELU_TRIPLE, tid, elem, ell);
            uint64_t e = rmod((uint64_t)dprime - (T.b0 + T.b1), ell);
            uint64_t d = rmod((s0[i] - T.a0) + (s1[i] - T.a1), ell);
            uint64_t xd0 = rmod(d * e + d * T.b0 + e * T.a0 + T.c0, ell);
            uint64_t xd1 = rmod(d * T.b1 + e * T.a1 + T.c1, ell);
            o0[i] = rmod(one_m2t * xd0 + (uint64_t)t * s0[i], ell);   /* unflip */
            o1[i] = rmod(one_m2t * xd1 + (uint64_t)t * s1[i], ell);
        }
        if (w0) memcpy(w0 + i * L, msg0, sizeof(uint64_t) * L);
        if (w1) memcpy(w1 + i * L, msg1, sizeof(uint64_t) * L);
        if (dprime_out) dprime_out[i] = (uint8_t)dprime;
    }
    return 0;
}

/* Steps 1-9 of the 1.0-style protocol over many elements with explicit
   randomness (row i: t[i], fy[i*L ..], r[i*L ..], z[i*L ..]); for the pins. */
int orc_drelu_b1_core_many(const orc_params *P, const uint64_t *s0, const uint64_t *s1,
                           const uint8_t *t, const uint32_t *fy, const uint64_t *r,
                           const uint64_t *z, size_t n, uint8_t *dprime)
{
    if (check_params_b1(P)) return -1;
    const int L = P->lx + 1;
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint64_t msg0[MAXL], msg1[MAXL];
        dprime[i] = (uint8_t)orc_drelu_b1_core(P, s0[i], s1[i], t[i], fy + i * L, r + i * L,
                                               z + i * L, msg0, msg1);
    }
    return 0;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Steps 1-9 of Alg. drelu over many elements with explicit randomness
 * (row i uses t[i], fy[i*L ..], r[i*L ..], z[i*L ..]); used by the brute-force
 * pins, which sweep t and the shares directly. */
int orc_drelu_core_many(const orc_params *P, const uint64_t *s0, const uint64_t *s1,
                        const uint8_t *t, const uint32_t *fy, const uint32_t *r,
                        const uint32_t *z, size_t n, uint8_t *dprime)
{
    if (check_params(P)) return -1;
    const int L = P->lx + 1;
    ORC_PARALLEL_FOR
    for (size_t i = 0; i < n; i++) {
        uint32_t msg0[MAXL], msg1[MAXL];
        dprime[i] = (uint8_t)orc_drelu_core(P, s0[i], s1[i], t[i], fy + i * L, r + i * L,
                                            z + i * L, msg0, msg1);
    }
    return 0;
}
