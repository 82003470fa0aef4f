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
  12     u32x4 tile parameters after default resolution
  28     u32  flags that select code (GENERIC, NO_AOT, INJECT_COMPILE_ERROR,
              INJECT_WAIT_TIMEOUT)

All little-endian.  Fields that a kernel does not use are zeroed, so requests
differing only there share an instantiation.

Default tile resolution (tile all zero, no cost model):
  update chain / grouped, bf16:   (3 = bf16 tensor-core panels, max(1, 128 // n16), 0, 0),
                                  n16 = n rounded up to a multiple of 16
  f64 or f32, n <= 4:             (2 = instance per thread, 128, 0, 0)
  grouped f32, n >= 17:           (5 = 4x4 register blocks, 1, 0, 0)
  f32, n >= 9:                    (6 = two rows per thread, max(1, 128 // ceil(n / 2)), 0, 0)
  otherwise:                      (1 = row per thread, ipb, 0, 0) with
                                  ipb = max(1, 256 // n) for n <= 32, max(1, 128 // n) above
  Eigen recurrence: (mapping, ipb, 0, 0); mapping 2 (two rows per thread)
      for f32 with n >= 2, else 1; ipb = max(1, 128 // tpi) with tpi =
      ceil(n / 2) or n threads per instance, lowered while the two shared
      buffers (rows padded to an odd number of 16-byte units, instances to 16
      bytes modulo 128 where a half-warp's rows would share banks) exceed
      96 KiB.
  LTimes: (TG, TZ, threads, (PIPE << 20) | (MODE << 16) | (R << 8) | S);
      orders 1, 4 are g-fast and 0, 2 z-fast; TG = 1 if neither in nor out
      is g-fast, 8 if one is g-fast and the other z-fast, else 32.
      f32 with m <= 128: TZ = 128 // TG; mode 5 (TMA-fed tcgen05, R 2, S 8,
      448 threads) with the largest PIPE in (4, 3, 2) whose shared memory
      fits 220 KiB, else mode 4 (R 2, S 8, 416 threads) if that fits.
      Otherwise CT = 64 columns, TZ = CT // TG; f64: R 1, S 9, threads
      64 * ceil(m / 9); f32: PIPE 1, R 2, S 12, threads 32 * ceil(m / 12).
  LPlusTimes: the LTimes default of the swapped problem (orders exchanged,
      m and d exchanged).
Expected variant: GENERIC flag -> generic; else update chain f64/f32 with
n in {4, 8, 16, 32}, default tile, AoT set enabled and neither NO_AOT nor
INJECT_COMPILE_ERROR -> aot; else jit.
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


G_FAST = (1, 4)
Z_FAST = (0, 2)


def _tc_smem(m, d, stages, tg, tz, lout, boxes):
    """Shared-memory bytes of the tensor-core LTimes kernel (restated from the
    documented layout): 1 KiB alignment slack; `boxes` TMA boxes of 128 x 32
    floats; per operand stage two 128 x 32 tf32 tiles in 16 groups of 1168
    bytes; L's hi and lo parts (moments padded to 16, directions to 32); the
    out box (m fastest: 128 rows of mp floats, mp a multiple of 4 with mp / 4
    odd; otherwise m rows of 128 / run runs, each run padded by 4 floats when
    it is at least 8 long, run = the box extent of out's fastest axis)."""
    np_, dp = -(-m // 16) * 16, -(-d // 32) * 32
    if lout in (3, 5):
        b = -(-m // 4)
        box = 128 * (4 * b if b % 2 else 4 * b + 4)
    else:
        run = tg if lout in (1, 4) else tz
        box = m * (128 // run) * (run + 4 if run >= 8 else run)
    return 1024 + boxes * 128 * 32 * 4 + stages * 2 * 16 * 1168 + 2 * np_ * dp * 4 + box * 4


def default_tile(kernel: int, dtype: int, n: int, layout_a: int = 0, layout_b: int = 0, m: int = 36,
                 d: int = 96) -> tuple:
    if kernel == K_EIGEN_RECURRENCE:
        # f32 with n >= 2: two rows per thread (mapping 2, tpi = ceil(n / 2)
        # threads per instance), else one (mapping 1, tpi = n);
        # max(1, 128 // tpi) instances per block, fewer while the two buffers
        # exceed 96 KiB; a row is an odd number of 16-byte units; an instance is
        # n rows, padded by 16-byte units to 16 bytes modulo 128 when two
        # instances read by one half-warp (threads 16k .. 16k + 15, thread t on
        # instance t // tpi) would start a multiple of 128 bytes apart
        es = 8 if dtype == F64 else 4
        mapping = 2 if dtype == F32 and n >= 2 else 1
        tpi = (n + 1) // 2 if mapping == 2 else n
        rp = ((-(-n * es // 16)) | 1) * 16 // es
        units = n * rp * es // 16
        collide = any((d * n * rp * es) % 128 == 0
                      for k in range(tpi) for d in range(1, (16 * k + 15) // tpi - (16 * k) // tpi + 1))
        ip = n * rp + ((1 - units) % 8) * (16 // es) if collide else n * rp
        ipb = max(1, 128 // tpi)
        while ipb > 1 and 2 * ipb * ip * es > 96 * 1024:
            ipb -= 1
        return (mapping, ipb, 0, 0)
    if kernel == K_UPDATE_CHAIN_GROUPED and dtype == F32 and n >= 17:
        return (5, 1, 0, 0)            # one large instance per block, 4x4 register blocks
    if kernel in (K_UPDATE_CHAIN, K_UPDATE_CHAIN_GROUPED):
        if dtype == BF16:
            return (3, max(1, 128 // (-(-n // 16) * 16)), 0, 0)
        if n <= 4:
            return (2, 128, 0, 0)
        if dtype == F32 and n >= 9:          # two rows of X per thread
            return (6, max(1, 128 // ((n + 1) // 2)), 0, 0)
        return (1, max(1, (256 if n <= 32 else 128) // n), 0, 0)
    if kernel == K_LPLUSTIMES:     # LTimes of the swapped problem
        return default_tile(K_LTIMES, dtype, n, layout_b, layout_a, d, m)
    if kernel == K_LTIMES:
        ct = 64
        gin, gout = layout_a in G_FAST, layout_b in G_FAST
        if not gin and not gout:
            tg = 1
        elif (gin and layout_b in Z_FAST) or (gout and layout_a in Z_FAST):
            tg = 8
        else:
            tg = 32
        if dtype == F32 and m <= 128:
            # tensor-core modes: 128 columns, 2 operand stages, 8 converter
            # warps; TMA-fed (mode 5) with the deepest box ring that fits in
            # 220 KiB of shared memory, else register producers (mode 4)
            for boxes in (4, 3, 2):
                if _tc_smem(m, d, 2, tg, 128 // tg, layout_b, boxes) <= 220 * 1024:
                    return (tg, 128 // tg, 32 * (6 + 8), (boxes << 20) | (5 << 16) | (2 << 8) | 8)
            if _tc_smem(m, d, 2, tg, 128 // tg, layout_b, 0) <= 220 * 1024:
                return (tg, 128 // tg, 32 * (5 + 8), (4 << 16) | (2 << 8) | 8)
        if dtype == F32:
            return (tg, ct // tg, 32 * (-(-m // 12)), (1 << 20) | (2 << 8) | 12)
        return (tg, ct // tg, ct * (-(-m // 9)), (1 << 8) | 9)
    raise ValueError("unknown kernel")


def canonical_key(kernel: int, dtype: int, n=0, layout_a=0, layout_b=0, m=0, d=0,
                  tile=(0, 0, 0, 0), flags=0) -> bytes:
    tile = tuple(tile)
    if kernel in (K_UPDATE_CHAIN, K_UPDATE_CHAIN_GROUPED, K_EIGEN_RECURRENCE):
        m = d = layout_b = 0
        if kernel in (K_UPDATE_CHAIN_GROUPED, K_EIGEN_RECURRENCE):
            layout_a = 0
    elif kernel in (K_LTIMES, K_LPLUSTIMES):
        n = 0
    if flags & FLAG_GENERIC:
        tile = (0, 0, 0, 0)            # the generic kernel has no tile template
    elif all(t == 0 for t in tile):
        tile = default_tile(kernel, dtype, n, layout_a, layout_b, m, d)
    return struct.pack("<HBBBBHHH4II", kernel, dtype, layout_a, layout_b, 0, n, m, d,
                       *tile, flags & KEY_FLAGS)


def expected_variant(kernel: int, dtype: int, n: int, tile=(0, 0, 0, 0), flags=0,
                     enable_aot_set=True) -> int:
    if flags & FLAG_GENERIC:
        return VARIANT_GENERIC
    if (kernel == K_UPDATE_CHAIN and dtype in (F64, F32) and n in AOT_SIZES
            and enable_aot_set and not (flags & (FLAG_NO_AOT | FLAG_INJECT_COMPILE_ERROR))
            and tuple(tile) in ((0, 0, 0, 0), default_tile(kernel, dtype, n))):
        return VARIANT_AOT
    return VARIANT_JIT
