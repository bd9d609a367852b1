"""Algorithmic work of the hot path, per element, for the roofline.

The fused DReLU/ReLU kernel is bound by integer issue, not by HBM: per element
it moves 32 bytes (l = 64: two input shares, two output shares) but executes
thousands of 32-bit integer operations.  This module fixes the count of
integer operations the protocol needs per element (the "algorithmic ops"),
step by step, so that achieved = ops x elements / time can be set against the
GPU's integer issue peak.  Counting rules (one op = one 32-bit integer
instruction a GPU thread must issue at minimum):

  Philox-4x32-10 block          10 rounds x (2 widening multiplies + 2 three-input XORs) = 40
  per message slot (lx+1 slots), both parties and the helper:
      window (Alg. newtrc2)     2 parties x 2 windows x (shift + mask)                   =  8
      pair sum (step 4)         2 parties x (add + mask)                                 =  4
      modulo switch (step 5)    P0 test + select, P1 add                                 =  3
      r_k, z_k from 128 bits    2 x 2 multiplies + 1 add                                 =  5
      masking (step 7)          3 Montgomery products x 5 (r to Montgomery form, 2 shares)= 15
      reshare (step 8)          2 x (add, compare, select)                               =  6
      P2 (step 9)               add mod p (3) + zero test and OR (2)                     =  5
  shuffle (step 6)              lx swaps x (index multiply + 2 loads + 2 stores)         = 5 lx
  flip (steps 1-2)              2 negations on 64/32-bit lanes                           =  6
  ReLU finish (Alg. relu)       triple completion, openings, 3 products, select:
                                40 ops on 64-bit lanes, 20 on 32-bit lanes
  DReLU finish (steps 10-11)    8 ops
Philox blocks per element: ceil((lx+1)/4) (t and shuffle) + (lx+1) (masks) +
3 (ReLU triple at l > 32; 2 at l <= 32) or 1 (DReLU reply).

The elementwise kernels (sharing, truncations, modulo switch) are HBM-bound;
their algorithmic bytes are the lanes read plus the lanes written.
"""
from __future__ import annotations

PHILOX_BLOCK_OPS = 40
SLOT_OPS = 8 + 4 + 3 + 5 + 15 + 6 + 5     # = 46


def philox_blocks(lx: int, ring_bits: int, relu: bool) -> int:
    L = lx + 1
    extra = (3 if ring_bits > 32 else 2) if relu else 1
    return (L + 3) // 4 + L + extra


def int_ops_per_element(lx: int, ring_bits: int, relu: bool = True) -> int:
    L = lx + 1
    finish = (40 if ring_bits > 32 else 20) if relu else 8
    return (philox_blocks(lx, ring_bits, relu) * PHILOX_BLOCK_OPS + L * SLOT_OPS + 5 * lx + 6
            + finish)


def hbm_bytes_per_element_relu(ring_bits: int) -> int:
    lane = 8 if ring_bits > 32 else 4
    return 4 * lane            # read [x]_0, [x]_1; write two output shares


def int_issue_peak_ops(sm_count: int = 152, sm_mhz: float = 2070.0) -> float:
    """Integer issue peak: each SM issues 4 warp instructions per clock (one
    per scheduler), i.e. 128 32-bit lane operations per clock when the ALU and
    FMA (IMAD) pipes are both fed.  Uses the maximum SM clock."""
    return sm_count * 4 * 32 * sm_mhz * 1e6
