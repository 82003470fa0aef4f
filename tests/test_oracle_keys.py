"""Pin of the key encoder against byte strings assembled by hand from the
documented 32-byte little-endian format (kernel u16, dtype u8, layout_a u8,
layout_b u8, pad u8, n u16, m u16, d u16, tile u32 x4, flags u32)."""
from oracle import keys as K


def test_hand_assembled_chain_key():
    # kernel 1, f64, row-major, n=8, default tile (1, 32, 0, 0) (one thread per
    # row, 256 / n instances per block), no flags
    expect = bytes.fromhex("0100" "00" "00" "00" "00" "0800" "0000" "0000"
                           "01000000" "20000000" "00000000" "00000000" "00000000")
    assert K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8) == expect


def test_hand_assembled_ltimes_key():
    # kernel 2, f32, in GZD(3), out ZGD(5), m=36, d=96, default tile
    # (1, 128, 448, (4 << 20) | (5 << 16) | (2 << 8) | 8): tensor cores fed by
    # TMA (mode 5), 4 TMA boxes, 2 operand stages, 8 converter warps (448 threads)
    expect = bytes.fromhex("0200" "01" "03" "05" "00" "0000" "2400" "6000"
                           "01000000" "80000000" "c0010000" "08024500" "00000000")
    assert K.canonical_key(K.K_LTIMES, K.F32, layout_a=3, layout_b=5, m=36, d=96) == expect


def test_generic_flag_drops_tile_and_keeps_flag():
    k = K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=8, tile=(1, 16, 0, 0), flags=K.FLAG_GENERIC)
    assert k[12:28] == bytes(16) and k[28:] == bytes([1, 0, 0, 0])


def test_golden_file_is_current():
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "tests", "golden", "keys.txt")) as f:
        before = f.read()
    lines = [l for l in before.splitlines() if not l.startswith("#")]
    for l in lines:
        f_ = l.split()
        k, dt, n, la, lb, m, d, t0, t1, t2, t3, fl = (int(v) for v in f_[:12])
        assert K.canonical_key(k, dt, n, la, lb, m, d, (t0, t1, t2, t3), fl).hex() == f_[12]
        assert K.expected_variant(k, dt, n, (t0, t1, t2, t3), fl) == int(f_[13])
