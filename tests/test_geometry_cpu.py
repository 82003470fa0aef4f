"""Shared-memory geometry of the Eigen recurrence kernels, on the CPU.

geometry.h is compiled for the host with g++ and its row pitch (eig_rp),
instance pitch (eig_ip) and buffer size (eig_smem) are checked against a
brute-force model of the shared-memory reads: thread t of a block works on
instance t // tpi (tpi = n threads per instance with one row per thread,
ceil(n / 2) with two), all threads of an instance read the same row (a
broadcast), and a warp's 16-byte loads are served per half-warp, where two
different addresses in the same 16-byte bank group (address // 16 mod 8)
cost an extra pass."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_08555_b300", "csrc", "kernels")

PROG = r"""
#include <cstdio>
#include <initializer_list>
#include "geometry.h"
int main() {
    for (int es : {4, 8})
        for (int rows : {1, 2})
            for (int n = 1; n <= 32; ++n)
                std::printf("%d %d %d %d %d %ld\n", es, rows, n, cjg::eig_rp(n, es), cjg::eig_ip(n, es, rows),
                            cjg::eig_smem(n, 3, es, rows));
    return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    d = tmp_path_factory.mktemp("geom")
    src, exe = d / "geom.cpp", d / "geom"
    src.write_text(PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    rows = {}
    for line in out.split("\n"):
        if line.strip():
            es, r, n, rp, ip, smem = (int(v) for v in line.split())
            rows[(es, r, n)] = (rp, ip, smem)
    assert len(rows) == 2 * 2 * 32
    return rows


def half_warp_collides(n, rows, pitch_bytes, threads=1024):
    """Brute force: does any half-warp of a `threads`-thread block read two
    different instance rows that fall in the same 16-byte bank group?"""
    tpi = -(-n // rows)
    for start in range(0, threads, 16):
        groups = {}
        for t in range(start, start + 16):
            addr = (t // tpi) * pitch_bytes          # row 0 of the thread's instance
            g = (addr // 16) % 8
            if g in groups and groups[g] != addr:
                return True
            groups[g] = addr
    return False


def max_instances_per_half_warp(n, rows, threads=1024):
    tpi = -(-n // rows)
    return max(len({t // tpi for t in range(s, s + 16)}) for s in range(0, threads, 16))


def test_row_pitch_is_an_odd_number_of_16_byte_units(table):
    for (es, _, n), (rp, _, _) in table.items():
        assert rp >= n and (rp * es) % 16 == 0 and (rp * es // 16) % 2 == 1


def test_instance_pitch_against_brute_force(table):
    for (es, r, n), (rp, ip, smem) in table.items():
        plain = n * rp * es
        got = ip * es
        assert smem == 2 * 3 * got
        assert got % 16 == 0 and plain <= got < plain + 128
        if half_warp_collides(n, r, plain):
            # padded to 16 bytes modulo 128; that removes every collision the
            # eight bank groups allow
            assert got % 128 == 16, (es, r, n)
            if max_instances_per_half_warp(n, r) <= 8:
                assert not half_warp_collides(n, r, got), (es, r, n)
        else:
            assert got == plain, (es, r, n)       # no padding where nothing collides


def test_known_cases(table):
    # f32, one row per thread: n = 8 (two instances per half-warp, 384-byte
    # pitch) is padded by one 16-byte unit; n = 16 (one instance per
    # half-warp) is not
    assert table[(4, 1, 8)][1] * 4 == 384 + 16
    assert table[(4, 1, 16)][1] * 4 == 16 * 20 * 4
    # f32, two rows per thread: n = 16 puts two instances in a half-warp
    assert table[(4, 2, 16)][1] * 4 == 16 * 20 * 4 + 16


LT_PROG = r"""
#include <cstdio>
#include <initializer_list>
#include "geometry.h"
int main() {
    for (int m : {1, 5, 16, 17, 36, 64, 100, 128})
        for (int d : {1, 31, 32, 33, 96, 128})
            for (int stages : {2, 3, 8})
                for (int tg : {1, 8, 32})
                    for (int lout = 0; lout < 6; ++lout)
                        for (int boxes : {0, 2, 4})
                            std::printf("%d %d %d %d %d %d %ld\n", m, d, stages, tg, lout, boxes,
                                        cjg::lt_tc_smem(m, d, stages, tg, 128 / tg, lout, boxes));
    return 0;
}
"""


def _tc_smem_model(m, d, stages, tg, tz, lout, boxes):
    """Shared-memory bytes of the tcgen05 LTimes kernel, summed buffer by
    buffer from the layout the kernel documents: 1 KiB of alignment slack;
    `boxes` TMA boxes of 128 x 32 floats; per operand stage two 128 x 32 tf32
    tiles (hi, lo) of 16 core-matrix groups of 1168 bytes (8 rows x 144-byte
    K-adjacent units, with the 16-byte pads); L's hi and lo parts with the
    moments padded to 16 and the directions to 32; the staged out box: for
    m fastest, 128 rows of mp floats (mp a multiple of 4 with mp / 4 odd),
    otherwise m rows of 128 / run runs, each padded by 4 floats when at
    least 8 long (run = the box extent of out's fastest axis)."""
    np_, dp = -(-m // 16) * 16, -(-d // 32) * 32
    if lout in (3, 5):
        b = -(-m // 4)
        box = 128 * (4 * b if b % 2 else 4 * b + 4)
    else:
        run = tg if lout in (1, 4) else tz
        box = m * (128 // run) * (run + 4 if run >= 8 else run)
    return 1024 + boxes * 128 * 32 * 4 + stages * 2 * 16 * 1168 + 2 * np_ * dp * 4 + box * 4


def test_tensor_core_ltimes_smem_matches_its_layout(tmp_path):
    """The tcgen05 LTimes kernel's shared-memory size in geometry.h equals the
    sum of its buffers as the kernel's layout describes them, over a grid of
    moments, directions, operand stages, column tiles, out orders and TMA
    boxes."""
    src, exe = tmp_path / "lt.cpp", tmp_path / "lt"
    src.write_text(LT_PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    lines = [l for l in out if l.strip()]
    assert len(lines) == 8 * 6 * 3 * 3 * 6 * 3
    for l in lines:
        m, d, stages, tg, lout, boxes, smem = (int(v) for v in l.split())
        assert _tc_smem_model(m, d, stages, tg, 128 // tg, lout, boxes) == smem, l


REG_PROG = r"""
#include <cstdio>
#include "geometry.h"
int main() {
    for (int w = 0; w <= 16; ++w) std::printf("%d %d\n", w, cjg::lt_tc_maxreg(w));
    return 0;
}
"""


def test_tensor_core_register_cap_fits_the_sub_partitions(tmp_path):
    """lt_tc_maxreg(w) is the per-thread register cap of a tcgen05 LTimes
    block of 5 + w warps (mode 4: w producer warps; mode 5: w converter warps
    plus the TMA warp).  The warps spread over the SM's four sub-partitions of
    16,384 registers, so the busiest holds ceil((5 + w) / 4) warps: the cap
    must fit there and be the largest multiple of 8 that does, or 255, the
    most a thread can hold, when that is smaller."""
    src, exe = tmp_path / "reg.cpp", tmp_path / "reg"
    src.write_text(REG_PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in (l for l in out if l.strip()):
        w, regs = (int(v) for v in line.split())
        busiest = -(-(5 + w) // 4)
        assert 0 < regs <= 255 and busiest * 32 * regs <= 16384
        # maximal: 255, or a multiple of 8 whose next multiple no longer fits
        assert regs == 255 or (regs % 8 == 0 and busiest * 32 * (regs + 8) > 16384)
        assert (5 + w) * 32 * regs <= 65536      # the whole block fits the SM's register file


M8_PROG = r"""
#include <cstdio>
#include "geometry.h"
int main() {
    for (int n = 8; n <= 64; ++n)
        std::printf("%d %d %d %d %d %ld\n", n, cjg::chain_m8_xti(n), cjg::chain_arow(n, 8, 4),
                    cjg::chain_threads(n, 8, 3), cjg::chain_pitch(n, 8, 4), cjg::chain_smem(n, 8, 3, 4));
    return 0;
}
"""


def test_four_by_eight_register_blocks_layout(tmp_path):
    """Mapping 8 (FP32, 4 x 8 register blocks): A rows padded to a multiple of
    8 columns; one instance's X^T holds (n padded to 8) rows of (n padded to
    4) + 4 floats and is padded to an odd number of 16-byte units (the copies
    a warp reads then start in different bank groups); threads are
    ceil(n/4) * ceil(n/8) per instance, rounded up to whole warps; shared
    memory is A's staging plus two copies of X^T (read one, write the
    other), per instance."""
    src, exe = tmp_path / "m8.cpp", tmp_path / "m8"
    src.write_text(M8_PROG)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in (l for l in out if l.strip()):
        n, xti, arow, threads, pitch, smem = (int(v) for v in line.split())
        nr, nc = -(-n // 4) * 4, -(-n // 8) * 8
        assert arow == nc
        assert xti in (nc * (nr + 4), nc * (nr + 4) + 4) and xti % 4 == 0 and (xti // 4) % 2 == 1
        assert threads == -(-(3 * (nr // 4) * (nc // 8)) // 32) * 32
        assert pitch >= n * nc and pitch % 4 == 0 and (pitch // 4) % 2 == 1
        assert smem == 3 * (pitch + 2 * xti) * 4
