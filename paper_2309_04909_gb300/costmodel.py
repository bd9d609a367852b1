"""Algorithmic work of the hot path, per element, for the roofline.

The fused DReLU/ReLU kernel is bound by the GPU's integer units, not by HBM:
per element it moves 32 bytes (l = 64: two input shares, two output shares)
but needs thousands of 32-bit integer operations, about a third of them
multiplications.  On GB300 integer multiplies (IMAD, IMAD.WIDE, IMAD.HI) run on
the 16-lane FMA-heavy pipe of each SM sub-partition, half the width of the
issue port, so the multiplier is the binding unit; the remaining operations
(XOR, add, shift, compare, select) go to the 16-lane ALU pipe.

Counting rules, per element, of what the protocol as specified needs (the
implementation may do less, e.g. by reusing a product across Philox blocks;
that shows up as a higher fraction of the roofline, not as less work):

  Philox-4x32-10 block   10 rounds x (2 widening 32x32->64 multiplies + 2 three-input XORs)
  per message slot (lx + 1 slots), both parties and the helper:
      window (Alg. newtrc2)     2 parties x 2 windows x (shift + mask)              8 ops
      pair sum (step 4)         2 parties x (add + mask)                            4
      modulo switch (step 5)    P0 test + select, P1 add                            3
      rho_k, z_k from 128 bits  2 x (high product of the low word + widening)       5 ops, 2x4 mul
      masking (step 7)          2 Montgomery products (wide, low, wide, cmp, sel)  10 ops, 2x5 mul
      reshare (step 8)          2 x (add, compare, select)                          6
      P2 (step 9)               add mod p (3) + zero test and OR (2)                5
  shuffle (step 6)    lx swaps x (index high-multiply + 2 loads + 2 stores)         5 lx, 2 lx mul
  flip (steps 1-2)    2 negations                                                   6
  ReLU finish         triple completion, openings, 5 ring products, select          40 ops (l>32) / 20
  DReLU finish        reply and unflip                                              8 ops
Philox blocks per element: ceil((lx+1)/4) (t and the shuffle) + (lx+1) (masks) +
3 (ReLU triple, l > 32; 2 at l <= 32) or 1 (DReLU reply).

"mul" counts multiplier lane-operations: a widening 32x32->64 product is 2, a
high 32-bit product (hi32(a b)) also 2, a low 32-bit product 1, a 64-bit low
product 4.  The high product's weight is measured: chains of it issue at
7.9 lanes per clock per sub-partition on GB300, the rate of widening products
(7.2 in Philox rounds), against 16.0 for low products.
"""
from __future__ import annotations

PHILOX_BLOCK_OPS = 40
PHILOX_BLOCK_MUL = 40             # 20 widening products
SLOT_OPS = 8 + 4 + 3 + 5 + 10 + 6 + 5     # = 41
SLOT_MUL = 8 + 10                          # draws + 2 Montgomery products


def philox_blocks(lx: int, ring_bits: int, relu: bool) -> int:
    L = lx + 1
    extra = (3 if ring_bits > 32 else 2) if relu else 1
    return (L + 3) // 4 + L + extra


def int_ops_per_element(lx: int, ring_bits: int, relu: bool = True) -> int:
    L = lx + 1
    finish = (40 if ring_bits > 32 else 20) if relu else 8
    return (philox_blocks(lx, ring_bits, relu) * PHILOX_BLOCK_OPS + L * SLOT_OPS + 5 * lx + 6
            + finish)


def mul_ops_per_element(lx: int, ring_bits: int, relu: bool = True) -> int:
    """Multiplier lane-operations per element (see module doc)."""
    L = lx + 1
    finish = (20 if ring_bits > 32 else 5) if relu else 0
    return (philox_blocks(lx, ring_bits, relu) * PHILOX_BLOCK_MUL + L * SLOT_MUL + 2 * lx
            + finish)


# The fused step of a linear layer followed by a ReLU adds, per element:
#   Beaver product    Philox blocks of the triple: 3 (l > 32; a0 b0 | c0 | a1 b1)
#                     or 2 (l <= 32); 6 ring products (c1, d e, d b0, e a0, d b1,
#                     e a1), each 4 multiplier ops at l > 32 (a 64-bit low product)
#                     or 1; 14 ring adds/subtracts/masks (2 ops each at l > 32)
#   truncations       2 shifts, 3 negations, 2 masks (2 ops each at l > 32)
def product_mul_ops_per_element(ring_bits: int) -> int:
    wide = ring_bits > 32
    return (3 if wide else 2) * PHILOX_BLOCK_MUL + 6 * (4 if wide else 1)


def product_int_ops_per_element(ring_bits: int) -> int:
    wide = ring_bits > 32
    w = 2 if wide else 1
    return ((3 if wide else 2) * PHILOX_BLOCK_OPS + 6 * (4 if wide else 1) + 14 * w + 7 * w)


def linear_relu_mul_ops_per_element(lx: int, ring_bits: int) -> int:
    return product_mul_ops_per_element(ring_bits) + mul_ops_per_element(lx, ring_bits, True)


def linear_relu_int_ops_per_element(lx: int, ring_bits: int) -> int:
    return product_int_ops_per_element(ring_bits) + int_ops_per_element(lx, ring_bits, True)


def mul_counts_split(lx: int, ring_bits: int, relu: bool = True, product: bool = False):
    """(widening, low, high) products per element: mul_counts with its single
    products split into low halves (Montgomery's q, ring cross terms) and high
    halves (the 64x32 draws' hi32(lo q), one per draw, and the shuffle's lx
    indices), which the multiplier may issue at different rates."""
    wide, single = mul_counts(lx, ring_bits, relu, product)
    high = 2 * (lx + 1) + lx
    return wide, single - high, high


def mul_counts(lx: int, ring_bits: int, relu: bool = True, product: bool = False):
    """(widening 32x32->64 products, single 32-bit products) per element, the
    split of the multiplier lane-operations above (a widening product is 2 of
    them): Philox 20 widening per block; per slot two 64x32 high products
    (1 widening + 1 single each) and two Montgomery products (2 widening + 1
    single each); lx single for the shuffle; a 64-bit ring product is 1
    widening + 2 single (l > 32) or 1 single."""
    L = lx + 1
    wide = philox_blocks(lx, ring_bits, relu) * 20 + L * 6
    single = L * 4 + lx
    if relu:
        if ring_bits > 32:
            wide, single = wide + 5, single + 10
        else:
            single += 5
    if product:
        if ring_bits > 32:
            wide, single = wide + 3 * 20 + 6, single + 12
        else:
            wide, single = wide + 2 * 20, single + 6
    return wide, single


def hbm_bytes_per_element_linear_relu(ring_bits: int, det_bits: int = 48) -> int:
    """Fused step: read x0, x1, y0, y1; write the ReLU and the deterministic
    truncation shares (det lanes 8 bytes when l - k > 32)."""
    lane = 8 if ring_bits > 32 else 4
    det = 8 if det_bits > 32 else 4
    return 6 * lane + 2 * det


def hbm_bytes_per_element_relu(ring_bits: int) -> int:
    lane = 8 if ring_bits > 32 else 4
    return 4 * lane            # read [x]_0, [x]_1; write two output shares


SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def int_issue_peak_ops(sm_count: int = SM_COUNT, sm_mhz: float = SM_MAX_MHZ) -> float:
    """Issue peak: 4 schedulers per SM each issue one warp instruction (32
    lanes) per clock."""
    return sm_count * 4 * 32 * sm_mhz * 1e6


def int_mul_peak_ops(sm_count: int = SM_COUNT, sm_mhz: float = SM_MAX_MHZ) -> float:
    """Integer-multiplier peak: 4 sub-partitions per SM, each with a 16-lane
    FMA-heavy pipe that executes IMAD-class instructions."""
    return sm_count * 4 * 16 * sm_mhz * 1e6


# ---------------------------------------------------------------------------
# The protocol's messages over the paper's networks (Sec. 6: three servers,
# LAN1 = 5 Gbps with 0.2 ms round-trip time, LAN2 = 1 Gbps / 0.6 ms, WAN =
# 100 Mbps / 40 ms).  A model, for comparing the GPU's time per call with the
# time the messages of Alg. drelu / Alg. relu need on those links; nothing
# here is measured.
# ---------------------------------------------------------------------------
PAPER_NETWORKS = {"LAN1": (5e9, 0.2e-3), "LAN2": (1e9, 0.6e-3), "WAN": (100e6, 40e-3)}


def round_bits(ell: int, lx: int, n: int, relu: bool):
    """Per round, the protocol bits each party sends and receives:
    [(sent[P0, P1, P2], received[P0, P1, P2]), ...] for the two rounds.
    Round 1: w_0 and w_1 ((lx + 1)^2 bits per element each, Alg. drelu step
    8) to P2; for ReLU also the openings [x]_j - [a]_j between P0 and P1 and
    the preprocessing message [c]_1 from P2 to P1, which depends on no input
    and so travels while P2's link out is otherwise idle.  Round 2: P2's
    reply, [DReLU']_1 to P1 (l bits), or for ReLU e = DReLU' - b to both."""
    w = n * (lx + 1) ** 2
    lane = n * ell
    sent1, recv1 = [w, w, 0], [0, 0, 2 * w]
    if relu:
        sent1 = [w + lane, w + lane, lane]
        recv1 = [lane, 2 * lane, 2 * w]
        sent2, recv2 = [0, 0, 2 * lane], [lane, lane, 0]
    else:
        sent2, recv2 = [0, 0, lane], [0, lane, 0]
    return [(sent1, recv1), (sent2, recv2)]


def network_seconds(ell: int, lx: int, n: int, relu: bool, bits_per_s: float,
                    rtt_s: float) -> float:
    """Time of the two rounds on links of bits_per_s each way per server
    (one full-duplex link per server, so a server's messages out share it,
    and so do its messages in), each round paying half the round-trip time:
    sum over rounds of rtt/2 + max over servers and directions of bits /
    bits_per_s."""
    t = 0.0
    for sent, recv in round_bits(ell, lx, n, relu):
        t += rtt_s / 2 + max(max(sent), max(recv)) / bits_per_s
    return t
