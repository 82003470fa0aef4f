"""Writes tests/golden/keys.txt from oracle/keys.py (the only source it calls).

Run: python tests/golden/make_golden.py
Each line: request fields, expected canonical key (hex) and expected variant.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import keys as K  # noqa: E402

REQUESTS = [
    # kernel, dtype, n, layout_a, layout_b, m, d, tile, flags
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 3, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 5, 1, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (0, 0, 0, 0), K.FLAG_GENERIC),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (0, 0, 0, 0), K.FLAG_NO_AOT),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (1, 16, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 32, 1, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 16, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 4, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F32, 64, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.BF16, 16, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 3, 36, 96, (0, 0, 0, 0), 0),        # unused fields zeroed
    (K.K_LTIMES, K.F64, 0, 0, 0, 36, 96, (0, 0, 0, 0), 0),
    (K.K_LTIMES, K.F64, 7, 3, 5, 36, 96, (0, 0, 0, 0), 0),               # n ignored
    (K.K_LTIMES, K.F32, 0, 5, 1, 36, 96, (0, 0, 0, 0), 0),
    (K.K_LTIMES, K.F64, 0, 2, 4, 36, 96, (0, 0, 0, 0), K.FLAG_GENERIC),
    (K.K_LTIMES, K.F32, 0, 1, 1, 36, 96, (32, 4, 192, (2 << 8) | 12), 0),
    (K.K_LTIMES, K.F32, 0, 0, 1, 64, 128, (0, 0, 0, 0), 0),             # tensor cores: fewer TMA boxes fit
    (K.K_LTIMES, K.F32, 0, 4, 3, 64, 128, (0, 0, 0, 0), 0),
    (K.K_LTIMES, K.F32, 0, 2, 4, 48, 100, (0, 0, 0, 0), 0),
    (K.K_LPLUSTIMES, K.F32, 0, 1, 2, 36, 96, (0, 0, 0, 0), 0),          # swapped: 96 rows, K = 36
    (K.K_LPLUSTIMES, K.F32, 0, 0, 0, 64, 128, (0, 0, 0, 0), 0),         # 128 rows
    (K.K_UPDATE_CHAIN_GROUPED, K.F64, 20, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_UPDATE_CHAIN_GROUPED, K.F32, 3, 1, 0, 0, 0, (0, 0, 0, 0), 0),  # layout forced 0
    (K.K_UPDATE_CHAIN_GROUPED, K.F32, 45, 0, 0, 0, 0, (0, 0, 0, 0), 0),  # one large instance per block
    (K.K_UPDATE_CHAIN, K.F64, 8, 0, 0, 0, 0, (0, 0, 0, 0), K.FLAG_INJECT_COMPILE_ERROR),
    (K.K_EIGEN_RECURRENCE, K.F64, 16, 1, 2, 36, 96, (0, 0, 0, 0), 0),   # unused fields zeroed
    (K.K_EIGEN_RECURRENCE, K.F32, 32, 0, 0, 0, 0, (0, 0, 0, 0), 0),
    (K.K_EIGEN_RECURRENCE, K.F64, 3, 0, 0, 0, 0, (0, 0, 0, 0), K.FLAG_GENERIC),
]


def main():
    path = os.path.join(ROOT, "tests", "golden", "keys.txt")
    with open(path, "w") as f:
        f.write("# Canonical instantiation keys (written by tests/golden/make_golden.py from oracle/keys.py).\n")
        f.write("# kernel dtype n layout_a layout_b m d t0 t1 t2 t3 flags key_hex variant(0 gen,1 aot,2 jit)\n")
        for (k, dt, n, la, lb, m, d, tile, fl) in REQUESTS:
            key = K.canonical_key(k, dt, n, la, lb, m, d, tile, fl).hex()
            var = K.expected_variant(k, dt, n, tile, fl)
            f.write(" ".join(str(v) for v in (k, dt, n, la, lb, m, d, *tile, fl, key, var)) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
