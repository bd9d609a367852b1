"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/bicoptor.h declares.  No compute calls."""
import ctypes
import os
import re

from paper_2309_04909_gb300 import _native

HEADER = os.path.join(_native.INCLUDE, "bicoptor.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bc_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("bc_share", "bc_trunc_prob", "bc_trunc_det", "bc_mod_switch", "bc_drelu", "bc_relu",
              "bc_reconstruct", "bc_mul_beaver", "bc_relu_batch"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    path = _native.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    # the binding's signature table covers the same set
    assert set(_native.SIGNATURES) == set(declared_symbols())


def test_host_only_helpers():
    import oracle as O
    lib = _native.lib()
    for lx in (1, 2, 7, 9, 14, 24, 31):
        assert lib.bc_prime_above(lx) == O.prime_above(lx)
    assert lib.bc_prime_above(0) == 0 and lib.bc_prime_above(32) == 0
    assert lib.bc_strerror(-1) == b"invalid argument"
    # argument checks that fail before touching the GPU
    assert lib.bc_create(None, 1, 0, None) == -1
    assert lib.bc_destroy(None) == -1


def test_costmodel_counts():
    from paper_2309_04909_gb300 import costmodel as C
    # (lx+1) mask blocks + ceil((lx+1)/4) shuffle blocks + triple blocks
    assert C.philox_blocks(24, 64, True) == 7 + 25 + 3
    assert C.philox_blocks(9, 32, False) == 3 + 10 + 1
    assert C.int_ops_per_element(24, 64) > C.int_ops_per_element(9, 32)
    # per slot: two 64x32 draws (widening + high product, 4 each) and two
    # Montgomery products (5 each); the shuffle's lx high products (2 each)
    assert C.mul_ops_per_element(24, 64) == 35 * 40 + 25 * 18 + 2 * 24 + 20
    w, lo, hi = C.mul_counts_split(24, 64, relu=True, product=True)
    assert (w, lo, hi) == (921, 72, 74)
    assert 2 * w + lo + 2 * hi == C.linear_relu_mul_ops_per_element(24, 64)


def test_key_bit_params():
    """Sec. 6.1's key bits: 5 + 26 bits with 2 fractional bits kept is lx = 7
    with the last 24 bits ignored (the paper's example); 7 + 0 keeps no
    fractional bit; windows that do not fit the ring are refused."""
    import pytest
    from paper_2309_04909_gb300 import Params
    p = Params.from_key_bits(64, 5, 26, 2)
    assert (p.ring_bits, p.lx, p.key_off) == (64, 7, 24)
    p = Params.from_key_bits(64, 7, 26, 0)
    assert (p.lx, p.key_off) == (7, 26)
    assert Params.from_key_bits(32, 9, 14, 0) == Params(32, 9, 14)
    for bad in ((64, 5, 26, 27), (64, 20, 26, 12), (32, 9, 14, 1), (64, 0, 0, 0)):
        with pytest.raises(ValueError):
            Params.from_key_bits(*bad)
