"""Writes tests/golden/keys.txt from oracle/keys.py (the only source it calls).

Run: python tests/golden/make_golden.py
Each line: request fields (every tile explicit, or GENERIC), expected
canonical key (hex) and expected variant.  The tiles below are request
inputs chosen by hand from the documented tile fields (cj.h); no rule for
choosing a tile enters the expected keys.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import keys as K  # noqa: E402

Z4 = (0, 0, 0, 0)


def lt_tile(tg, tz, threads, mode, r, s, pipe=0):
    """LTimes tile field 3: (PIPE << 20) | (MODE << 16) | (R << 8) | S."""
    return (tg, tz, threads, (pipe << 20) | (mode << 16) | (r << 8) | s)


REQUESTS = [
    # kernel, dtype, n, layout_a, layout_b, m, d, tile, flags
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (1, 16, 0, 0), K.FLAG_NO_AOT),
    (K.K_UPDATE_CHAIN, K.F64, 3, 0, 0, 0, 0, (2, 128, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 5, 1, 0, 0, 0, (1, 51, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, Z4, K.FLAG_GENERIC),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (1, 32, 0, 16), K.FLAG_GENERIC),   # generic drops the tile
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (4, 2, 0, 0), K.FLAG_NO_AOT),
    (K.K_UPDATE_CHAIN, K.F64, 32, 1, 0, 0, 0, (1, 8, 0, 0), K.FLAG_NO_AOT),
    (K.K_UPDATE_CHAIN, K.F64, 12, 0, 0, 0, 0, (1, 4, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 16, 0, 0, 0, 0, (6, 16, 0, 0), K.FLAG_NO_AOT),
    (K.K_UPDATE_CHAIN, K.F32, 7, 1, 0, 0, 0, (2, 64, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 64, 0, 0, 0, 0, (6, 4, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 24, 0, 0, 0, 0, (5, 2, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.BF16, 16, 0, 0, 0, 0, (3, 8, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 12, 0, 3, 36, 96, (1, 21, 0, 0), 0),          # unused fields zeroed
    (K.K_LTIMES, K.F64, 0, 0, 0, 36, 96, lt_tile(1, 64, 256, 0, 1, 9), 0),
    (K.K_LTIMES, K.F64, 7, 3, 5, 36, 96, lt_tile(1, 64, 256, 0, 1, 9), 0),   # n ignored
    (K.K_LTIMES, K.F64, 0, 1, 0, 36, 96, lt_tile(8, 8, 128, 1, 2, 8), 0),    # FP64 mma.sync
    (K.K_LTIMES, K.F32, 0, 5, 1, 36, 96, lt_tile(32, 4, 448, 5, 2, 8, 4), 0),
    (K.K_LTIMES, K.F64, 0, 2, 4, 36, 96, Z4, K.FLAG_GENERIC),
    (K.K_LTIMES, K.F32, 0, 1, 1, 36, 96, lt_tile(32, 4, 192, 0, 2, 12), 0),
    (K.K_LTIMES, K.F32, 0, 0, 1, 64, 128, lt_tile(8, 16, 448, 5, 2, 8, 2), 0),
    (K.K_LTIMES, K.F32, 0, 4, 3, 64, 128, lt_tile(32, 4, 416, 4, 2, 8), 0),
    (K.K_LTIMES, K.F32, 0, 2, 4, 48, 100, lt_tile(8, 16, 448, 5, 2, 8, 3), 0),
    (K.K_LTIMES, K.F32, 0, 3, 3, 36, 96, lt_tile(1, 128, 448, 5, 2, 8, 4), K.FLAG_INJECT_WAIT_TIMEOUT),
    (K.K_LPLUSTIMES, K.F32, 0, 1, 2, 36, 96, lt_tile(8, 16, 416, 4, 2, 8), 0),   # swapped: 96 rows, K = 36
    (K.K_LPLUSTIMES, K.F32, 0, 0, 0, 64, 128, lt_tile(1, 128, 416, 4, 2, 8), 0),  # 128 rows
    (K.K_LPLUSTIMES, K.F64, 0, 4, 2, 36, 96, lt_tile(8, 8, 704, 0, 1, 9), 0),
    (K.K_UPDATE_CHAIN_GROUPED, K.F64, 20, 0, 0, 0, 0, (1, 12, 0, 0), 0),
    (K.K_UPDATE_CHAIN_GROUPED, K.F32, 3, 1, 0, 0, 0, (2, 128, 0, 0), 0),    # layout forced 0
    (K.K_UPDATE_CHAIN_GROUPED, K.F32, 45, 0, 0, 0, 0, (5, 1, 0, 0), 0),
    (K.K_UPDATE_CHAIN_GROUPED, K.BF16, 40, 0, 0, 0, 0, (3, 2, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (1, 32, 0, 0), K.FLAG_INJECT_COMPILE_ERROR),
    (K.K_EIGEN_RECURRENCE, K.F64, 16, 1, 2, 36, 96, (1, 8, 0, 0), 0),       # unused fields zeroed
    (K.K_EIGEN_RECURRENCE, K.F32, 32, 0, 0, 0, 0, (2, 8, 0, 0), 0),
    (K.K_EIGEN_RECURRENCE, K.F32, 9, 0, 0, 0, 0, (1, 14, 0, 0), 0),
    (K.K_EIGEN_RECURRENCE, K.F64, 3, 0, 0, 0, 0, Z4, K.FLAG_GENERIC),
]


def main():
    path = os.path.join(ROOT, "tests", "golden", "keys.txt")
    with open(path, "w") as f:
        f.write("# Canonical instantiation keys (written by tests/golden/make_golden.py from oracle/keys.py).\n")
        f.write("# Every request names its tile (or GENERIC); none leaves the tile to the library.\n")
        f.write("# kernel dtype n layout_a layout_b m d t0 t1 t2 t3 flags key_hex variant(0 gen,1 aot,2 jit)\n")
        for (k, dt, n, la, lb, m, d, tile, fl) in REQUESTS:
            key = K.canonical_key(k, dt, n, la, lb, m, d, tile, fl).hex()
            var = K.expected_variant(k, dt, n, tile_left_to_library=False, flags=fl)
            f.write(" ".join(str(v) for v in (k, dt, n, la, lb, m, d, *tile, fl, key, var)) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
