"""The network model of the protocol's messages (costmodel.round_bits,
network_seconds): its bit counts agree with the counters the library
reports for the same call (the fused kernel's bc_get_comm, checked on the
GPU elsewhere; here against the closed forms of Alg. drelu step 8 and
Alg. relu), and the times follow from them by hand."""
import pytest

from paper_2309_04909_gb300 import costmodel as C


def test_round_bits_match_the_protocol():
    n, ell, lx = 1000, 64, 7
    (s1, r1), (s2, r2) = C.round_bits(ell, lx, n, relu=False)
    assert s1 == [64_000, 64_000, 0] and r1 == [0, 0, 128_000]     # (lx+1)^2 = 64 bits each
    assert s2 == [0, 0, 64_000] and r2 == [0, 64_000, 0]           # [DReLU']_1 to P1
    (s1, r1), (s2, r2) = C.round_bits(ell, lx, n, relu=True)
    assert sum(s1) == sum(r1) and sum(s2) == sum(r2)               # every bit sent is received
    assert s1 == [128_000, 128_000, 64_000] and r1 == [64_000, 128_000, 128_000]
    assert s2 == [0, 0, 128_000] and r2 == [64_000, 64_000, 0]
    # the totals per direction are those of the library's counters (relu_comm):
    # 2 (lx+1)^2 + 5 l bits per element for ReLU, 2 (lx+1)^2 + l for DReLU
    assert sum(s1) + sum(s2) == n * (2 * 64 + 5 * 64)
    (a, _), (b, _) = C.round_bits(ell, lx, n, relu=False)
    assert sum(a) + sum(b) == n * (2 * 64 + 64)


def test_network_seconds_by_hand():
    bw, rtt = C.PAPER_NETWORKS["LAN1"]
    # DReLU, 10^6 elements, lx = 7: P2 takes in 2 x 64 Mbit, then sends 64 Mbit
    t = C.network_seconds(64, 7, 10**6, False, bw, rtt)
    assert t == pytest.approx(2 * 0.1e-3 + 128e6 / 5e9 + 64e6 / 5e9)
    # ReLU: 128 Mbit on P0's, P1's and P2's busiest direction in round 1, then
    # P2 sends e to both (128 Mbit)
    t = C.network_seconds(64, 7, 10**6, True, bw, rtt)
    assert t == pytest.approx(2 * 0.1e-3 + 2 * 128e6 / 5e9)
    # one element: latency only, to within a microsecond
    assert C.network_seconds(64, 7, 1, True, bw, rtt) == pytest.approx(rtt, abs=1e-6)
    # WAN is 50x slower per bit than LAN1
    assert (C.network_seconds(64, 24, 10**6, True, *C.PAPER_NETWORKS["WAN"]) - 40e-3) == \
        pytest.approx(50 * (C.network_seconds(64, 24, 10**6, True, bw, rtt) - 0.2e-3))
