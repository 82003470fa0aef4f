// geometry.h -- shared-memory pitches and block shapes.  Used by the kernels
// (compiled by nvcc ahead of time and by NVRTC at run time) and by the host
// launch code, so that both sides agree on every byte offset.  No includes.
#ifndef CJ_GEOMETRY_H
#define CJ_GEOMETRY_H

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define CJ_HD __host__ __device__
#else
#define CJ_HD
#endif

namespace cjg {

// Update chain, one thread per row (mapping 1): pitch in elements of one
// instance's A in shared memory.  At least nn, a whole number of 16-byte
// units, and an odd number of them so consecutive instances start in
// different bank groups (their threads read different addresses at once).
CJ_HD constexpr int row_pitch(int nn, int esize) {
    return ((((nn * esize + 15) / 16) | 1) * 16) / esize;
}

// Update chain, one thread per instance (mapping 2): each thread reads its
// own instance, so the pitch is odd (in elements) to spread 32 threads over
// 32 banks.
CJ_HD constexpr int inst_pitch(int nn) { return nn | 1; }

// Threads per block of the update chain kernels: mapping 2 one thread per
// instance, mapping 4 one warp per 8 rows, mapping 3 one warp per 16 rows
// (padded), mapping 5 one thread per 4x4 block, mapping 8 one thread per 4x8
// block (rows padded to 4, columns to 8), mapping 6 one thread per two rows,
// mapping 1 one thread per row.
CJ_HD constexpr int chain_threads(int n, int mapping, int ipb) {
    return mapping == 7   ? 128
           : mapping == 8 ? ((ipb * ((n + 3) / 4) * ((n + 7) / 8) + 31) / 32) * 32
           : mapping == 2 ? ipb
           : mapping == 6 ? ((ipb * ((n + 1) / 2) + 31) / 32) * 32
           : mapping == 5 ? ((ipb * ((n + 3) / 4) * ((n + 3) / 4) + 31) / 32) * 32
           : mapping == 4 ? ipb * (n / 8) * 32
           : mapping == 3 ? ipb * ((n + 15) / 16) * 32
                          : ((ipb * n + 31) / 32) * 32;
}

// Rows of X kept in shared memory (instead of registers) above this size.
CJ_HD constexpr int chain_reg_rows_max(int esize) { return esize == 8 ? 32 : 48; }

// Row length of A_b in shared memory: mappings 1, 5 and 6 in FP32 pad each
// row to a multiple of 4 so a thread reads A with 16-byte vectors (one
// shared-memory load per four fused multiply-adds per row of X the thread
// owns), mapping 8 to a multiple of 8 (its column blocks); every other
// mapping keeps rows of n.
CJ_HD constexpr int chain_arow(int n, int mapping, int esize) {
    return (mapping == 8 && esize == 4)                                           ? (n + 7) / 8 * 8
           : ((mapping == 1 || mapping == 5 || mapping == 6) && esize == 4) ? (n + 3) / 4 * 4
                                                                            : n;
}

// Mapping 8 (FP32): one copy of an instance's X^T (it keeps two), (n padded
// to 8) rows of pitch (n padded to 4) + 4, then padded to an odd number of
// 16-byte units, so that the copies a warp reads start in different bank
// groups.
CJ_HD constexpr int chain_m8_xti(int n) {
    return ((n + 7) / 8 * 8) * ((n + 3) / 4 * 4 + 4) / 4 % 2 ? ((n + 7) / 8 * 8) * ((n + 3) / 4 * 4 + 4)
                                                             : ((n + 7) / 8 * 8) * ((n + 3) / 4 * 4 + 4) + 4;
}

// Elements between consecutive staged instances of the specialized kernels.
CJ_HD constexpr int chain_pitch(int n, int mapping, int esize) {
    return mapping == 2 ? inst_pitch(n * n) : row_pitch(n * chain_arow(n, mapping, esize), esize);
}

// Per-thread pitch of X rows kept in shared memory (odd: conflict-free).
CJ_HD constexpr int xrow_pitch(int n) { return n | 1; }

// Bytes of dynamic shared memory of the specialized update chain kernel.
CJ_HD constexpr long chain_smem(int n, int mapping, int ipb, int esize) {
    return mapping == 7
        ? 128L * ((n + 15) / 16 * 16) * 2 + (long)((n + 15) / 16 * 16) * ((n + 15) / 16 * 16) * 2
        : mapping == 2
        ? (long)ipb * inst_pitch(n * n) * esize
        : mapping == 5
        ? (long)ipb * chain_pitch(n, 5, esize) * esize + (long)ipb * ((n + 3) / 4 * 4) * ((n + 3) / 4 * 4 + 4) * esize
        : mapping == 8   // A, then two copies of X^T (chain_m8_xti elements each) per instance
        ? (long)ipb * chain_pitch(n, 8, esize) * esize + 2L * ipb * chain_m8_xti(n) * esize
        : (long)ipb * chain_pitch(n, mapping, esize) * esize +
              (mapping == 1 && n > chain_reg_rows_max(esize)
                   ? (long)chain_threads(n, 1, ipb) * xrow_pitch(n) * esize
               : mapping == 6 && n > 32 ? 2L * chain_threads(n, 6, ipb) * xrow_pitch(n) * esize
                                        : 0L);
}

// Eigen recurrence (both kernels): two buffers of M per instance.  Rows are
// a whole, odd number of 16-byte units: 16-byte aligned for vector reads of a
// row, and consecutive rows start in different bank groups.
CJ_HD constexpr int eig_rp(int n, int esize) {
    return ((n * esize + 15) / 16 | 1) * 16 / esize;
}
// Thread t works on instance t / tpi (tpi threads per instance: n with one
// row per thread, ceil(n / 2) with two) and reads one row of that instance's
// M per load, the same row as the instance's other threads (a broadcast).  A
// warp's 16-byte shared-memory loads are served per half-warp, so two
// instances whose rows sit in the same half-warp's load collide when their
// addresses differ by a multiple of 128 bytes (same banks).  Half-warp k
// spans instances 16k / tpi .. (16k + 15) / tpi, a pattern that repeats every
// tpi.
CJ_HD constexpr bool eig_collide(int tpi, int pitch_bytes) {
    for (int k = 0; k < tpi; ++k)
        for (int d = 1; d <= (16 * k + 15) / tpi - (16 * k) / tpi; ++d)
            if ((d * pitch_bytes) % 128 == 0) return true;
    return false;
}
// Instance pitch for `rows` rows of M per thread: n rows of eig_rp; where
// instances collide, padded by whole 16-byte units to 16 bytes modulo 128,
// which puts the instances of a half-warp in different banks (up to 8).
CJ_HD constexpr int eig_ip(int n, int esize, int rows = 1) {
    return eig_collide((n + rows - 1) / rows, n * eig_rp(n, esize) * esize)
               ? n * eig_rp(n, esize) + (((1 - n * eig_rp(n, esize) * esize / 16) % 8 + 8) % 8) * (16 / esize)
               : n * eig_rp(n, esize);
}
CJ_HD constexpr long eig_smem(int n, int ipb, int esize, int rows = 1) {
    return 2L * ipb * eig_ip(n, esize, rows) * esize;
}

// Generic update chain: A pitch uses row_pitch; each thread keeps its row of
// X and of the product in shared memory with pitch xrow_pitch(n).
CJ_HD constexpr long chain_generic_smem(int n, int ipb, int threads, int esize) {
    return (long)ipb * row_pitch(n * n, esize) * esize + 2L * threads * xrow_pitch(n) * esize;
}

// LTimes: L is kept transposed, [d][m] with m padded to whole moment groups
// of S and to a 16-byte multiple.
CJ_HD constexpr int lt_mpitch(int mpad, int esize) { return ((mpad * esize + 15) / 16) * 16 / esize; }
// Column tile pitch: CT plus 16 bytes (mode 2: plus 8 elements, so the four
// k-rows of an mma fragment fall in different banks).
CJ_HD constexpr int lt_cpitch(int ct, int esize, int mode = 0) { return ct + (mode == 2 ? 8 : 16 / esize); }
// pipe = 1: two tile buffers; mode 2: a second copy of L^T (tf32 remainder).
CJ_HD constexpr long lt_smem(int m, int s, int d, int ct, int esize, int pipe = 0, int mode = 0) {
    return ((mode == 2 ? 2L : 1L) * d * lt_mpitch((m + s - 1) / s * s, esize) +
            (pipe ? 2L : 1L) * (long)(m > d ? m : d) * lt_cpitch(ct, esize, mode)) *
           esize;
}
// Direct kernel (mode 3, s moments per thread, 0 = all): L^T padded to whole
// moment groups, plus one out box.
CJ_HD constexpr int lt_direct_mpad(int m, int s) {
    return (s == 0 || s >= m) ? (m + 3) / 4 * 4 : (m + s - 1) / s * s;
}
CJ_HD constexpr long lt_direct_smem(int m, int d, int ct, int esize, int s = 0) {
    return ((long)d * lt_mpitch(lt_direct_mpad(m, s), esize) + (long)m * lt_cpitch(ct, esize)) * esize;
}
// tcgen05 kernel (mode 4, FP32): 128-column tiles, MMA N = moments padded to
// 16, K = directions padded to 32; `stages` operand tiles (tf32 hi and lo,
// 128 x 32 each), L's hi and lo parts, one out box, 1 KB alignment slack.
CJ_HD constexpr int lt_tc_np(int m) { return (m + 15) / 16 * 16; }
CJ_HD constexpr int lt_tc_dp(int d) { return (d + 31) / 32 * 32; }
// Registers per thread for one block of 5 + nprod warps per SM (nprod counts
// the TMA warp in mode 5): the warps are spread over the SM's four
// sub-partitions of 16K registers each, so the fullest one holds
// ceil(warps / 4) of them (multiples of 8, at most 255).
CJ_HD constexpr int lt_tc_maxreg(int nprod) {
    return 16384 / (32 * ((5 + nprod + 3) / 4)) / 8 * 8 > 255 ? 255 : 16384 / (32 * ((5 + nprod + 3) / 4)) / 8 * 8;
}
// Operand tile of one stage (128 columns x 32 directions, tf32): K-adjacent
// core matrices LBO bytes apart, 8-row groups SBO bytes apart (both padded
// by 16 bytes off a multiple of 128 so writes spread over all banks).
constexpr unsigned LT_TC_A_LBO = 144, LT_TC_A_SBO = 8 * 144 + 16, LT_TC_A_BYTES = 16 * LT_TC_A_SBO;
// Staged out box: runs of `run` floats along out's faster column axis,
// padded by 4 floats when that spreads a warp's writes over all banks.
CJ_HD constexpr int lt_tc_runp(int run) { return run >= 8 ? run + 4 : run; }
// m-fastest out: one box row of mp floats per column, mp / 4 odd.
CJ_HD constexpr int lt_tc_mp(int m) { return (m + 3) / 4 % 2 ? (m + 3) / 4 * 4 : (m + 3) / 4 * 4 + 4; }
// Shared memory of the tcgen05 kernel; tg, tz and out's storage order fix
// the box (out's fastest axis: z for orders 0 and 2, g for 1 and 4, m for 3
// and 5).
CJ_HD constexpr long lt_tc_box(int m, int tg, int tz, int lout) {
    return lout == 3 || lout == 5 ? 128L * lt_tc_mp(m)
                                  : (long)m * (128 / (lout == 1 || lout == 4 ? tg : tz)) *
                                        lt_tc_runp(lout == 1 || lout == 4 ? tg : tz);
}
// rawst: TMA boxes of `in` (128 columns x 32 directions) ahead of the operand
// ring (mode 5; 0 in mode 4).
CJ_HD constexpr long lt_tc_smem(int m, int d, int stages, int tg, int tz, int lout, int rawst = 0) {
    return 1024L + (long)rawst * 128 * 32 * 4 + (long)stages * 2 * LT_TC_A_BYTES + 2L * lt_tc_np(m) * lt_tc_dp(d) * 4 +
           lt_tc_box(m, tg, tz, lout) * 4;
}
CJ_HD constexpr long lt_generic_smem(int m, int d, int cols, int esize) {
    return ((long)m * d + (long)d * cols) * esize;
}

// Mass operator (mass.cuh): an element owns M x M threads, M = max(D, Q);
// shared memory holds B1 (Q x D) and two buffers of M^dim values per element.
CJ_HD constexpr int mass_m(int D, int Q) { return D > Q ? D : Q; }
// form 2 (2-D, one thread per element, every stage in registers): epb threads.
CJ_HD constexpr int mass_threads(int D, int Q, int epb, int form = 0) {
    return form == 2 ? (epb + 31) / 32 * 32 : ((epb * mass_m(D, Q) * mass_m(D, Q) + 31) / 32) * 32;
}
CJ_HD constexpr int mass_b_elems(int D, int Q) { return Q * D; }
// form 1 (the persistent kernel): two stages of every element's x (D^dim)
// and op (Q^dim) values besides; form 2: B1 only.
CJ_HD constexpr long mass_smem(int dim, int D, int Q, int epb, int esize, int form = 0) {
    return form == 2 ? (long)mass_b_elems(D, Q) * esize
                     : ((long)mass_b_elems(D, Q) +
                        2L * epb * (dim == 2 ? mass_m(D, Q) * mass_m(D, Q) : mass_m(D, Q) * mass_m(D, Q) * mass_m(D, Q)) +
                        (form ? 2L * epb * (dim == 2 ? D * D + Q * Q : D * D * D + Q * Q * Q) : 0L)) *
                           esize;
}
// Form 2 keeps an element's D x Q first-stage values and its D x D result in
// registers: allowed while D Q + D^2 <= 80.
CJ_HD constexpr bool mass_thread_ok(int dim, int D, int Q) { return dim == 2 && D * Q + D * D <= 80; }

}  // namespace cjg

#endif
