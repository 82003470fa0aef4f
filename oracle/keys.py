"""Canonical instantiation keys and the expected dispatch choice -- TEST INFRASTRUCTURE.

A restatement, written from the documented key format, of what the library
must produce for a specialization request.  The paper's runtime looks an
instantiation up by {mangled template name, non-type template values, type
strings} (Sec. 4, Algorithm 1, first step); our key is the byte image of the
same information for a fixed set of kernel templates:

  offset size field
  0      u16  kernel id (1 update chain, 2 LTimes, 3 grouped update chain,
                          4 LPlusTimes, 5 Eigen recurrence)
  2      u8   dtype (0 f64, 1 f32, 2 bf16 operands / f32 state)
  3      u8   layout_a (chain: 0 row-major, 1 column-major; LTimes: in order 0..5)
  4      u8   layout_b (LTimes: out order 0..5; else 0)
  5      u8   reserved, 0
  6      u16  n (chain / Eigen matrix size; else 0)
  8      u16  m (LTimes moments; else 0)
  10     u16  d (LTimes directions; else 0)
  12     u32x4 tile parameters (the instantiation's tile template arguments)
  28     u32  flags that select code (GENERIC, NO_AOT, INJECT_COMPILE_ERROR,
              INJECT_WAIT_TIMEOUT)

All little-endian.  Fields that a kernel does not use are zeroed, so requests
differing only there share an instantiation.

What this module fixes is the contract only: the byte format, the zeroing of
unused fields, the flag semantics and the variant rule.  Which tile the
library picks for a request that leaves the tile to it is a performance
choice, not part of the contract, so it is not restated here: a key is
formed from a tile that is already explicit (the request's own, or the one
the library reports it resolved to), and a request with GENERIC keys the
generic kernel, which has no tile.

Variant rule (Sec. 2: an explicit specialization compiled ahead of time is
used instead of compiling the same instantiation at run time):
  GENERIC flag                                    -> generic
  update chain, f64 or f32, n in {4, 8, 16, 32}, the ahead-of-time set
  enabled, the tile left to the library, neither NO_AOT nor
  INJECT_COMPILE_ERROR                            -> aot
  anything else                                   -> jit
An explicit tile equal to the one an ahead-of-time kernel was built with is
the same instantiation (the same key), so it is served by that kernel too;
the tests check this through the handle cache rather than by naming the
ahead-of-time tiles here.
"""
from __future__ import annotations

import struct

K_UPDATE_CHAIN = 1
K_LTIMES = 2
K_UPDATE_CHAIN_GROUPED = 3
K_LPLUSTIMES = 4
K_EIGEN_RECURRENCE = 5

F64, F32, BF16 = 0, 1, 2

FLAG_GENERIC = 1
FLAG_NO_AOT = 2
FLAG_INJECT_COMPILE_ERROR = 0x100
FLAG_INJECT_WAIT_TIMEOUT = 0x200
KEY_FLAGS = FLAG_GENERIC | FLAG_NO_AOT | FLAG_INJECT_COMPILE_ERROR | FLAG_INJECT_WAIT_TIMEOUT

AOT_SIZES = (4, 8, 16, 32)

VARIANT_GENERIC, VARIANT_AOT, VARIANT_JIT = 0, 1, 2

_KEY_FORMAT = "<HBBBBHHH4II"


def canonical_key(kernel: int, dtype: int, n=0, layout_a=0, layout_b=0, m=0, d=0,
                  tile=(0, 0, 0, 0), flags=0) -> bytes:
    """The 32-byte key of an instantiation.  `tile` must be explicit unless
    `flags` has GENERIC (the generic kernel has no tile template)."""
    tile = tuple(int(t) for t in tile)
    if len(tile) != 4:
        raise ValueError("a tile has four fields")
    if kernel in (K_UPDATE_CHAIN, K_UPDATE_CHAIN_GROUPED, K_EIGEN_RECURRENCE):
        m = d = layout_b = 0
        if kernel in (K_UPDATE_CHAIN_GROUPED, K_EIGEN_RECURRENCE):
            layout_a = 0
    elif kernel in (K_LTIMES, K_LPLUSTIMES):
        n = 0
    else:
        raise ValueError("unknown kernel")
    if flags & FLAG_GENERIC:
        tile = (0, 0, 0, 0)
    elif all(t == 0 for t in tile):
        raise ValueError("a key is formed from an explicit (resolved) tile")
    return struct.pack(_KEY_FORMAT, kernel, dtype, layout_a, layout_b, 0, n, m, d, *tile, flags & KEY_FLAGS)


def parse_key(key: bytes) -> dict:
    """The fields of a 32-byte key (the inverse of canonical_key's packing)."""
    if len(key) != 32:
        raise ValueError("a key is 32 bytes")
    kernel, dtype, la, lb, pad, n, m, d, t0, t1, t2, t3, flags = struct.unpack(_KEY_FORMAT, key)
    return dict(kernel=kernel, dtype=dtype, layout_a=la, layout_b=lb, reserved=pad, n=n, m=m, d=d,
                tile=(t0, t1, t2, t3), flags=flags)


def expected_variant(kernel: int, dtype: int, n: int, tile_left_to_library: bool, flags=0,
                     enable_aot_set=True) -> int:
    if flags & FLAG_GENERIC:
        return VARIANT_GENERIC
    if (kernel == K_UPDATE_CHAIN and dtype in (F64, F32) and n in AOT_SIZES and enable_aot_set
            and tile_left_to_library and not (flags & (FLAG_NO_AOT | FLAG_INJECT_COMPILE_ERROR))):
        return VARIANT_AOT
    return VARIANT_JIT
