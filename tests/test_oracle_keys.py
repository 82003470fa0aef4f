"""Pins of the key encoder (oracle/keys.py) against byte strings assembled by
hand from the documented 32-byte little-endian format (kernel u16, dtype u8,
layout_a u8, layout_b u8, pad u8, n u16, m u16, d u16, tile u32 x4, flags
u32), and of the variant rule against the statement of Sec. 2 (an explicit
ahead-of-time specialization is used instead of compiling the same
instantiation)."""
import os

import pytest

from oracle import keys as K


def test_hand_assembled_chain_key():
    # kernel 1, f64, row-major, n=8, tile (1, 32, 0, 0), no flags
    expect = bytes.fromhex("0100" "00" "00" "00" "00" "0800" "0000" "0000"
                           "01000000" "20000000" "00000000" "00000000" "00000000")
    assert K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8, tile=(1, 32, 0, 0)) == expect


def test_hand_assembled_ltimes_key():
    # kernel 2, f32, in GZD(3), out ZGD(5), m=36, d=96, tile
    # (1, 128, 448, (4 << 20) | (5 << 16) | (2 << 8) | 8)
    expect = bytes.fromhex("0200" "01" "03" "05" "00" "0000" "2400" "6000"
                           "01000000" "80000000" "c0010000" "08024500" "00000000")
    tile = (1, 128, 448, (4 << 20) | (5 << 16) | (2 << 8) | 8)
    assert K.canonical_key(K.K_LTIMES, K.F32, layout_a=3, layout_b=5, m=36, d=96, tile=tile) == expect


def test_hand_assembled_flag_and_zeroed_fields():
    # kernel 3 (grouped), bf16, n=40: layout_a, layout_b, m and d are not
    # template arguments of this kernel and are zeroed; NO_AOT is kept
    expect = bytes.fromhex("0300" "02" "00" "00" "00" "2800" "0000" "0000"
                           "03000000" "02000000" "00000000" "00000000" "02000000")
    got = K.canonical_key(K.K_UPDATE_CHAIN_GROUPED, K.BF16, n=40, layout_a=1, layout_b=3, m=36, d=96,
                          tile=(3, 2, 0, 0), flags=K.FLAG_NO_AOT)
    assert got == expect


def test_ltimes_key_ignores_n_and_chain_key_ignores_m_d():
    t = (1, 64, 256, (1 << 8) | 9)
    assert (K.canonical_key(K.K_LTIMES, K.F64, n=7, m=36, d=96, tile=t) ==
            K.canonical_key(K.K_LTIMES, K.F64, m=36, d=96, tile=t))
    assert (K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=5, m=36, d=96, layout_b=4, tile=(1, 8, 0, 0)) ==
            K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=5, tile=(1, 8, 0, 0)))


def test_generic_flag_drops_tile_and_keeps_flag():
    k = K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8, tile=(1, 16, 0, 0), flags=K.FLAG_GENERIC)
    assert k[12:28] == bytes(16) and k[28:] == bytes([1, 0, 0, 0])


def test_flags_outside_the_key_are_dropped():
    a = K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8, tile=(1, 16, 0, 0), flags=0x4000 | K.FLAG_NO_AOT)
    assert a[28:] == bytes([2, 0, 0, 0])


def test_a_key_needs_an_explicit_tile():
    with pytest.raises(ValueError):
        K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8)
    with pytest.raises(ValueError):
        K.canonical_key(9, K.F64, n=8, tile=(1, 1, 0, 0))


def test_parse_inverts_the_packing():
    t = (8, 16, 448, 0x250208)
    key = K.canonical_key(K.K_LTIMES, K.F32, layout_a=0, layout_b=1, m=64, d=128, tile=t,
                          flags=K.FLAG_INJECT_WAIT_TIMEOUT)
    f = K.parse_key(key)
    assert (f["kernel"], f["dtype"], f["layout_a"], f["layout_b"], f["reserved"], f["n"], f["m"], f["d"],
            f["tile"], f["flags"]) == (2, 1, 0, 1, 0, 0, 64, 128, t, 0x200)


def test_variant_rule():
    ev = K.expected_variant
    # ahead-of-time sizes, tile left to the library, f64/f32 update chain
    for n in (4, 8, 16, 32):
        for dt in (K.F64, K.F32):
            assert ev(K.K_UPDATE_CHAIN, dt, n, True) == K.VARIANT_AOT
            assert ev(K.K_UPDATE_CHAIN, dt, n, True, enable_aot_set=False) == K.VARIANT_JIT
            assert ev(K.K_UPDATE_CHAIN, dt, n, True, flags=K.FLAG_NO_AOT) == K.VARIANT_JIT
            assert ev(K.K_UPDATE_CHAIN, dt, n, True, flags=K.FLAG_INJECT_COMPILE_ERROR) == K.VARIANT_JIT
            assert ev(K.K_UPDATE_CHAIN, dt, n, True, flags=K.FLAG_GENERIC) == K.VARIANT_GENERIC
    # not in the set: other sizes, bf16, other kernels
    assert ev(K.K_UPDATE_CHAIN, K.F64, 12, True) == K.VARIANT_JIT
    assert ev(K.K_UPDATE_CHAIN, K.BF16, 16, True) == K.VARIANT_JIT
    assert ev(K.K_UPDATE_CHAIN_GROUPED, K.F64, 8, True) == K.VARIANT_JIT
    assert ev(K.K_EIGEN_RECURRENCE, K.F64, 8, True) == K.VARIANT_JIT
    assert ev(K.K_LTIMES, K.F64, 0, True) == K.VARIANT_JIT
    assert ev(K.K_LTIMES, K.F64, 0, False, flags=K.FLAG_GENERIC) == K.VARIANT_GENERIC


def test_golden_file_is_current():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "tests", "golden", "keys.txt")) as f:
        lines = [l for l in f.read().splitlines() if not l.startswith("#")]
    assert len(lines) >= 30
    for l in lines:
        f_ = l.split()
        k, dt, n, la, lb, m, d, t0, t1, t2, t3, fl = (int(v) for v in f_[:12])
        assert (t0, t1, t2, t3) != (0, 0, 0, 0) or fl & K.FLAG_GENERIC, l
        assert K.canonical_key(k, dt, n, la, lb, m, d, (t0, t1, t2, t3), fl).hex() == f_[12]
        assert K.expected_variant(k, dt, n, False, fl) == int(f_[13])
