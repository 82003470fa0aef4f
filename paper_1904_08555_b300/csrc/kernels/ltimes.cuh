// ltimes.cuh -- Kripke's LTimes contraction with run-time storage orders
// (Sec. 5.2, Listings kripold / kripnew):
//     out[m][g][z] = sum_{d<D} L[m][d] * in[d][g][z]
// on logical indices.  A storage order lists the axes (x, g, z) slowest to
// fastest, x = d for `in` and m for `out`:
//     0 XGZ, 1 XZG, 2 GXZ, 3 GZX, 4 ZXG, 5 ZGX.
// The specialized kernel takes both orders, M, D and the tile as template
// arguments, so every index computation below folds to constants; the generic
// kernel takes M, D and all six strides at run time with one fixed thread
// mapping.  No includes besides geometry.h.
#ifndef CJ_LTIMES_CUH
#define CJ_LTIMES_CUH
#include "geometry.h"

// Bounded waits of the tcgen05 kernels that expired (each block counts once).
__device__ unsigned int cj_wait_timeouts;

namespace cj {

__device__ __forceinline__ double lt_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float lt_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Slot (0 slowest .. 2 fastest) of axis a (0 = x, 1 = g, 2 = z) in order lay.
__host__ __device__ constexpr int lt_pos(int lay, int a) {
    return (lay == 0) ? (a == 0 ? 0 : a == 1 ? 1 : 2)     // X G Z
         : (lay == 1) ? (a == 0 ? 0 : a == 1 ? 2 : 1)     // X Z G
         : (lay == 2) ? (a == 0 ? 1 : a == 1 ? 0 : 2)     // G X Z
         : (lay == 3) ? (a == 0 ? 2 : a == 1 ? 0 : 1)     // G Z X
         : (lay == 4) ? (a == 0 ? 1 : a == 1 ? 2 : 0)     // Z X G
                      : (a == 0 ? 2 : a == 1 ? 1 : 0);    // Z G X
}

// Axis stored at slot s of order lay.
__host__ __device__ constexpr int lt_axis(int lay, int s) {
    return lt_pos(lay, 0) == s ? 0 : lt_pos(lay, 1) == s ? 1 : 2;
}

// Move an (EX x TG x TZ) box between global memory (order LAY, extents
// EX, G, Z, box origin (0, g0, z0)) and shared memory laid out as
// s[x * CP + gl * TZ + zl].  Consecutive threads walk the box in storage
// order, so each warp touches consecutive global addresses.
template <class T, int LAY, int EX, int TG, int TZ, int CP, int NT, bool LOAD, bool ACC = false>
__device__ __forceinline__ void lt_box(T* __restrict__ g, T* s, long long G, long long Z,
                                       long long g0, long long z0, int tid) {
    constexpr int a0 = lt_axis(LAY, 0), a1 = lt_axis(LAY, 1), a2 = lt_axis(LAY, 2);
    constexpr int b0 = a0 == 0 ? EX : a0 == 1 ? TG : TZ;
    constexpr int b1 = a1 == 0 ? EX : a1 == 1 ? TG : TZ;
    constexpr int b2 = a2 == 0 ? EX : a2 == 1 ? TG : TZ;
    constexpr int TOTAL = b0 * b1 * b2;
    const long long ext[3] = {EX, G, Z};
    long long st[3];
    st[a2] = 1;
    st[a1] = ext[a2];
    st[a0] = ext[a2] * ext[a1];
    const long long gbase = g0 * st[1] + z0 * st[2];
#pragma unroll 4
    for (int e = tid; e < TOTAL; e += NT) {
        const int i2 = e % b2;
        const int i1 = (e / b2) % b1;
        const int i0 = e / (b2 * b1);
        int c[3];
        c[a0] = i0;
        c[a1] = i1;
        c[a2] = i2;
        const int x = c[0], gl = c[1], zl = c[2];
        const bool ok = (g0 + gl < G) && (z0 + zl < Z);
        const long long goff = gbase + (long long)x * st[0] + (long long)gl * st[1] + (long long)zl * st[2];
        T* sp = s + x * CP + gl * TZ + zl;
        if (LOAD) *sp = ok ? g[goff] : T(0);
        else if (ok) g[goff] = ACC ? g[goff] + *sp : *sp;
    }
}

// FP64 tensor-core contraction of one staged tile (MODE 1): warp w owns the
// 8*R columns starting at 8*R*w and every moment, in blocks of 8.  For the
// k-block of directions 4kb..4kb+3 it multiplies the (8 columns x 4 d) slice
// of the staged `in` tile (mma A operand: a[col][d] at lane 4*col + d) by
// the (4 d x 8 m) slice of L^T (B operand: b[d][m] at lane 4*m + d) into an
// 8 x 8 (column x moment) accumulator (c[col][m] at lane 4*col + m/2,
// component m%2).
__device__ __forceinline__ void lt_dmma(double (&d)[2], double a, double b) {
    asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(d[0]), "+d"(d[1])
        : "d"(a), "d"(b));
}

// 3xTF32 tensor-core step (MODE 2, FP32): a = a_hi + a_lo with both parts
// rounded to tf32; a*b ~ a_hi*b_hi + a_hi*b_lo + a_lo*b_hi (the dropped
// a_lo*b_lo term is ~2^-22 relative), accumulated in FP32 by mma.sync
// m16n8k8.  Fragment layouts (PTX ISA, m16n8k8 .tf32): A a0 (row g, col t),
// a1 (row g+8, col t), a2 (row g, col t+4), a3 (row g+8, col t+4); B b0
// (k t, n g), b1 (k t+4, n g); accumulator c0,c1 (row g, cols 2t, 2t+1),
// c2,c3 (row g+8, cols 2t, 2t+1); g = lane/4, t = lane%4.
__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Asynchronous variant of the box load (cp.async, one element per copy):
// out-of-range elements are zero-filled (source size 0), nothing is read.
template <class T, int LAY, int EX, int TG, int TZ, int CP, int NT>
__device__ __forceinline__ void lt_box_async(const T* __restrict__ g, T* s, long long G, long long Z,
                                             long long g0, long long z0, int tid) {
    constexpr int a0 = lt_axis(LAY, 0), a1 = lt_axis(LAY, 1), a2 = lt_axis(LAY, 2);
    constexpr int b0 = a0 == 0 ? EX : a0 == 1 ? TG : TZ;
    constexpr int b1 = a1 == 0 ? EX : a1 == 1 ? TG : TZ;
    constexpr int b2 = a2 == 0 ? EX : a2 == 1 ? TG : TZ;
    constexpr int TOTAL = b0 * b1 * b2;
    const long long ext[3] = {EX, G, Z};
    long long st[3];
    st[a2] = 1;
    st[a1] = ext[a2];
    st[a0] = ext[a2] * ext[a1];
    const long long gbase = g0 * st[1] + z0 * st[2];
#pragma unroll 4
    for (int e = tid; e < TOTAL; e += NT) {
        const int i2 = e % b2;
        const int i1 = (e / b2) % b1;
        const int i0 = e / (b2 * b1);
        int c[3];
        c[a0] = i0;
        c[a1] = i1;
        c[a2] = i2;
        const int x = c[0], gl = c[1], zl = c[2];
        const bool ok = (g0 + gl < G) && (z0 + zl < Z);
        const T* src = ok ? g + gbase + (long long)x * st[0] + (long long)gl * st[1] + (long long)zl * st[2] : g;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(s + x * CP + gl * TZ + zl);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"((int)sizeof(T)),
                     "r"(ok ? (int)sizeof(T) : 0)
                     : "memory");
    }
}
__device__ __forceinline__ void lt_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lt_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Persistent kernel: L^T stays in shared memory; each block loops over
// (g, z) tiles: stage the in box, contract, stage and store the out box.
// MODE 0: FMA pipe, each thread R columns x S moments.  MODE 1 (FP64 only,
// S = 8, D a multiple of 4): FP64 tensor cores, each warp 8R columns x all
// moments.  PIPE 1: two tile buffers; the next tile's box is loaded with
// cp.async while the current one is contracted.  ACC 1: out += result
// (LPlusTimes accumulates into its output).
template <class T, int M, int D, int LIN, int LOUT, int TG, int TZ, int NT, int R, int S, int MODE = 0,
          int PIPE = 0, int ACC = 0>
__global__ void __launch_bounds__(NT)
ltimes(const T* __restrict__ L, const T* __restrict__ in, T* __restrict__ out, long long G, long long Z) {
    constexpr int CT = TG * TZ;
    constexpr int MG = (M + S - 1) / S;   // moment groups (the last may be partial)
    constexpr int MP = cjg::lt_mpitch(MG * S, (int)sizeof(T));
    constexpr int CP = cjg::lt_cpitch(CT, (int)sizeof(T), MODE);
    constexpr int QG = CT / R;   // column groups
    static_assert(MODE != 0 || (CT % R == 0 && QG * MG == NT), "tile does not cover the block");
    static_assert(MODE != 1 || (sizeof(T) == 8 && S == 8 && D % 4 == 0 && CT % (8 * R) == 0 &&
                                (CT / (8 * R)) * 32 == NT), "tensor-core tile does not cover the block");
    static_assert(MODE != 2 || (sizeof(T) == 4 && S == 8 && R == 1 && D % 8 == 0 && CT % 16 == 0 &&
                                (CT / 16) * 32 == NT), "3xTF32 tile does not cover the block");
    extern __shared__ __align__(16) unsigned char cj_smem[];
    constexpr int XR = M > D ? M : D;        // rows of a tile buffer
    T* sL = reinterpret_cast<T*>(cj_smem);   // [D][MP], L transposed
    T* sX0 = sL + D * MP;                     // [D][CP] in tile, then [M][CP] out tile
    T* sX1 = sX0 + XR * CP;                   // second buffer (PIPE)
    T* sLlo = sX0 + (PIPE ? 2 : 1) * XR * CP; // MODE 2: tf32 remainder of L^T
    const int tid = threadIdx.x;
    for (int e = tid; e < MP * D; e += NT) {
        const int m = e / D, d = e - m * D;
        const T v = m < M ? L[e] : T(0);
        if constexpr (MODE == 2) {
            const unsigned hi = to_tf32((float)v);
            sL[d * MP + m] = __uint_as_float(hi);
            sLlo[d * MP + m] = __uint_as_float(to_tf32((float)v - __uint_as_float(hi)));
        } else {
            sL[d * MP + m] = v;
        }
    }
    const long long ntg = (G + TG - 1) / TG, ntz = (Z + TZ - 1) / TZ;
    const long long ntiles = ntg * ntz;
    const int qg = tid % QG, sg = tid / QG;
    const int q0 = qg * R, m0 = sg * S;
    if (PIPE && (long long)blockIdx.x < ntiles) {
        const long long t0 = blockIdx.x;
        lt_box_async<T, LIN, D, TG, TZ, CP, NT>(in, sX0, G, Z, (t0 / ntz) * TG, (t0 % ntz) * TZ, tid);
    }
    if (PIPE) lt_async_commit();
    int buf = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
        const long long g0 = (t / ntz) * TG, z0 = (t % ntz) * TZ;
        T* sX = (PIPE && buf) ? sX1 : sX0;
        __syncthreads();   // the other buffer's previous contents are no longer read
        if (PIPE) {
            const long long tn = t + gridDim.x;
            if (tn < ntiles)
                lt_box_async<T, LIN, D, TG, TZ, CP, NT>(in, buf ? sX0 : sX1, G, Z, (tn / ntz) * TG,
                                                        (tn % ntz) * TZ, tid);
            lt_async_commit();
            lt_async_wait<1>();   // this tile's copies (all but the newest group) are done
        } else {
            lt_box<T, LIN, D, TG, TZ, CP, NT, true>(const_cast<T*>(in), sX, G, Z, g0, z0, tid);
        }
        __syncthreads();
        if constexpr (MODE == 2) {
            const int lane = tid & 31, g = lane >> 2, t = lane & 3;
            const int q0 = (tid >> 5) * 16;
            float acc[MG][4];
#pragma unroll
            for (int nb = 0; nb < MG; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;
#pragma unroll 2
            for (int kb = 0; kb < D / 8; ++kb) {
                const float* x0 = reinterpret_cast<const float*>(sX) + (8 * kb + t) * CP + q0 + g;
                const float* x4 = x0 + 4 * CP;
                const float av[4] = {x0[0], x0[8], x4[0], x4[8]};
                unsigned ahi[4], alo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ahi[i] = to_tf32(av[i]);
                    alo[i] = to_tf32(av[i] - __uint_as_float(ahi[i]));
                }
                const float* l0 = reinterpret_cast<const float*>(sL) + (8 * kb + t) * MP + g;
                const float* r0 = reinterpret_cast<const float*>(sLlo) + (8 * kb + t) * MP + g;
#pragma unroll
                for (int nb = 0; nb < MG; ++nb) {
                    const unsigned bh0 = __float_as_uint(l0[8 * nb]), bh1 = __float_as_uint(l0[4 * MP + 8 * nb]);
                    const unsigned bl0 = __float_as_uint(r0[8 * nb]), bl1 = __float_as_uint(r0[4 * MP + 8 * nb]);
                    mma_tf32_1688(acc[nb], alo, bh0, bh1);
                    mma_tf32_1688(acc[nb], ahi, bl0, bl1);
                    mma_tf32_1688(acc[nb], ahi, bh0, bh1);
                }
            }
            __syncthreads();
#pragma unroll
            for (int nb = 0; nb < MG; ++nb)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = 8 * nb + 2 * t + (i & 1);
                    const int q = q0 + g + (i >= 2 ? 8 : 0);
                    if (M % 8 == 0 || m < M) sX[m * CP + q] = acc[nb][i];
                }
            __syncthreads();
            lt_box<T, LOUT, M, TG, TZ, CP, NT, false, ACC != 0>(out, sX, G, Z, g0, z0, tid);
            continue;
        }
        if constexpr (MODE == 1) {
            const int lane = tid & 31, r = lane >> 2, t = lane & 3;
            const int c0 = (tid >> 5) * 8 * R;
            double acc[R][MG][2];
#pragma unroll
            for (int cb = 0; cb < R; ++cb)
#pragma unroll
                for (int nb = 0; nb < MG; ++nb) acc[cb][nb][0] = acc[cb][nb][1] = 0.0;
#pragma unroll 2
            for (int kb = 0; kb < D / 4; ++kb) {
                double a[R], b[MG];
#pragma unroll
                for (int cb = 0; cb < R; ++cb) a[cb] = sX[(4 * kb + t) * CP + c0 + 8 * cb + r];
#pragma unroll
                for (int nb = 0; nb < MG; ++nb) b[nb] = sL[(4 * kb + t) * MP + 8 * nb + r];
#pragma unroll
                for (int cb = 0; cb < R; ++cb)
#pragma unroll
                    for (int nb = 0; nb < MG; ++nb) lt_dmma(acc[cb][nb], a[cb], b[nb]);
            }
            __syncthreads();
#pragma unroll
            for (int cb = 0; cb < R; ++cb)
#pragma unroll
                for (int nb = 0; nb < MG; ++nb)
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int m = 8 * nb + 2 * t + i;
                        if (M % 8 == 0 || m < M) sX[m * CP + c0 + 8 * cb + r] = acc[cb][nb][i];
                    }
            __syncthreads();
            lt_box<T, LOUT, M, TG, TZ, CP, NT, false, ACC != 0>(out, sX, G, Z, g0, z0, tid);
            continue;
        }
        T acc[R][S];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int s = 0; s < S; ++s) acc[r][s] = T(0);
#pragma unroll 4
        for (int d = 0; d < D; ++d) {
            T xv[R], lv[S];
#pragma unroll
            for (int r = 0; r < R; ++r) xv[r] = sX[d * CP + q0 + r];
#pragma unroll
            for (int s = 0; s < S; ++s) lv[s] = sL[d * MP + m0 + s];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int s = 0; s < S; ++s) acc[r][s] = lt_fma(lv[s], xv[r], acc[r][s]);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (M % S == 0 || m0 + s < M)
#pragma unroll
                for (int r = 0; r < R; ++r) sX[(m0 + s) * CP + q0 + r] = acc[r][s];
        __syncthreads();
        lt_box<T, LOUT, M, TG, TZ, CP, NT, false, ACC != 0>(out, sX, G, Z, g0, z0, tid);
    }
    if (PIPE) lt_async_wait<0>();
}

// Direct FP32 kernel (MODE 3): no staging of `in`.  A block owns a TG x TZ
// box of (g, z) columns; thread t owns R consecutive columns in the order of
// `in`'s faster column axis and reads its columns straight from global memory
// (coalesced across the warp; 16-byte vectors along d when d is fastest),
// accumulating S moments (S = 0: all M) in registers against 16-byte
// broadcast reads of L^T; threads of one column group that own different
// moment groups reread the same `in` values from L1.  When `out` orders its
// column axes like `in` (the same column axis
// faster), each thread stores its columns straight from registers (coalesced,
// or 16-byte vectors along m when m is fastest); otherwise the out box goes
// through shared memory to be stored coalesced.
template <class T, int M, int D, int LIN, int LOUT, int TG, int TZ, int NT, int R, int S = 0, int ACC = 0>
__global__ void __launch_bounds__(NT)
ltimes_direct(const T* __restrict__ L, const T* __restrict__ in, T* __restrict__ out, long long G, long long Z) {
    constexpr int CT = TG * TZ;
    constexpr int SM_ = (S == 0 || S >= M) ? ((M + 3) / 4) * 4 : S;   // moments per thread
    constexpr int MG = (M + SM_ - 1) / SM_;                            // moment groups
    constexpr int MP = cjg::lt_mpitch(MG * SM_, (int)sizeof(T));
    constexpr int CP = cjg::lt_cpitch(CT, (int)sizeof(T));
    constexpr int M4 = SM_ / 4;
    constexpr int QG = CT / R;                                         // column groups
    static_assert(SM_ % 4 == 0 && QG * MG == NT, "tile does not cover the block");
    static_assert(sizeof(T) == 4 && MP % 4 == 0, "direct mode is FP32");
    // faster column axis of each tensor: g if g comes after z in its order
    constexpr bool G_FASTER = lt_pos(LIN, 1) > lt_pos(LIN, 2);
    constexpr bool OUT_G_FASTER = lt_pos(LOUT, 1) > lt_pos(LOUT, 2);
    constexpr bool D_FAST = lt_pos(LIN, 0) == 2;
    constexpr bool M_FAST = lt_pos(LOUT, 0) == 2;
    constexpr bool DIRECT_OUT = G_FASTER == OUT_G_FASTER;
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sL = reinterpret_cast<T*>(cj_smem);   // [D][MP], L transposed, zero-padded
    T* sO = sL + D * MP;                      // [M][CP] out box (staged stores)
    const int tid = threadIdx.x;
    for (int e = tid; e < MP * D; e += NT) {
        const int m = e / D, d = e - m * D;
        sL[d * MP + m] = m < M ? L[e] : T(0);
    }
    const long long ext[3] = {D, G, Z};
    long long st[3], so[3];
    st[lt_axis(LIN, 2)] = 1;
    st[lt_axis(LIN, 1)] = ext[lt_axis(LIN, 2)];
    st[lt_axis(LIN, 0)] = ext[lt_axis(LIN, 2)] * ext[lt_axis(LIN, 1)];
    const long long exo[3] = {M, G, Z};
    so[lt_axis(LOUT, 2)] = 1;
    so[lt_axis(LOUT, 1)] = exo[lt_axis(LOUT, 2)];
    so[lt_axis(LOUT, 0)] = exo[lt_axis(LOUT, 2)] * exo[lt_axis(LOUT, 1)];
    const long long ntg = (G + TG - 1) / TG, ntz = (Z + TZ - 1) / TZ;
    const long long ntiles = ntg * ntz;
    const int cg = tid % QG, m0 = (tid / QG) * SM_;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long g0 = (t / ntz) * TG, z0 = (t % ntz) * TZ;
        long long off[R], ooff[R];
        int sidx[R];
        bool ok[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int c = cg * R + r;
            const int gl = G_FASTER ? c % TG : c / TZ;
            const int zl = G_FASTER ? c / TG : c % TZ;
            ok[r] = (g0 + gl < G) && (z0 + zl < Z);
            off[r] = ok[r] ? (g0 + gl) * st[1] + (z0 + zl) * st[2] : 0;
            ooff[r] = ok[r] ? (g0 + gl) * so[1] + (z0 + zl) * so[2] : 0;
            sidx[r] = gl * TZ + zl;
        }
        if (!DIRECT_OUT || t == blockIdx.x) __syncthreads();   // sL ready; previous out box stored
        T acc[R][SM_];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < SM_; ++m) acc[r][m] = T(0);
        auto step = [&](int d, const T (&x)[R]) {
            const float4* lrow = reinterpret_cast<const float4*>(sL + d * MP + m0);
#pragma unroll
            for (int m4 = 0; m4 < M4; ++m4) {
                const float4 lv = lrow[m4];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[r][4 * m4 + 0] = lt_fma(lv.x, x[r], acc[r][4 * m4 + 0]);
                    acc[r][4 * m4 + 1] = lt_fma(lv.y, x[r], acc[r][4 * m4 + 1]);
                    acc[r][4 * m4 + 2] = lt_fma(lv.z, x[r], acc[r][4 * m4 + 2]);
                    acc[r][4 * m4 + 3] = lt_fma(lv.w, x[r], acc[r][4 * m4 + 3]);
                }
            }
        };
        if constexpr (D_FAST && D % 4 == 0) {
#pragma unroll 2
            for (int d = 0; d < D; d += 4) {
                float4 xv[R];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    xv[r] = ok[r] ? __ldg(reinterpret_cast<const float4*>(in + off[r] + d)) : make_float4(0, 0, 0, 0);
                T x0[R], x1[R], x2[R], x3[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    x0[r] = xv[r].x;
                    x1[r] = xv[r].y;
                    x2[r] = xv[r].z;
                    x3[r] = xv[r].w;
                }
                step(d, x0);
                step(d + 1, x1);
                step(d + 2, x2);
                step(d + 3, x3);
            }
        } else {
#pragma unroll 4
            for (int d = 0; d < D; ++d) {
                T x[R];
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = ok[r] ? __ldg(in + off[r] + d * st[0]) : T(0);
                step(d, x);
            }
        }
        if constexpr (DIRECT_OUT) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!ok[r]) continue;
                T* o = out + ooff[r];
                if constexpr (M_FAST && M % SM_ == 0) {
#pragma unroll
                    for (int m4 = 0; m4 < M4; ++m4) {
                        float4 v = make_float4(acc[r][4 * m4], acc[r][4 * m4 + 1], acc[r][4 * m4 + 2], acc[r][4 * m4 + 3]);
                        float4* p = reinterpret_cast<float4*>(o + m0) + m4;
                        if (ACC) {
                            const float4 w = *p;
                            v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
                        }
                        *p = v;
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < SM_; ++m) {
                        if (M % SM_ != 0 && m0 + m >= M) break;
                        T* p = o + (m0 + m) * so[0];
                        *p = ACC ? *p + acc[r][m] : acc[r][m];
                    }
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int m = 0; m < SM_; ++m)
                    if (M % SM_ == 0 || m0 + m < M) sO[(m0 + m) * CP + sidx[r]] = acc[r][m];
            __syncthreads();
            lt_box<T, LOUT, M, TG, TZ, CP, NT, false, ACC != 0>(out, sO, G, Z, g0, z0, tid);
        }
    }
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (MODE 4, FP32 in and out).  The contraction of
// a 128-column tile is the GEMM D[col][m] = sum_d in[d][col] L[m][d] with the
// 128 columns as the MMA's M dimension, the moments (padded to NP, a
// multiple of 16) as N and the directions (padded to DP, a multiple of 32)
// as K.  Each product runs as three TF32 products, in_lo L_hi + in_hi L_lo +
// in_hi L_hi (x = x_hi + x_lo, both parts rounded to tf32; the dropped
// in_lo L_lo term is below FP32 rounding), on tcgen05.mma kind::tf32 with
// the FP32 accumulator in tensor memory.
//
// Roles (warp w): w 0-3 epilogue (TMEM lanes 32w..32w+31 = tile columns),
// w 4 allocates TMEM and one lane issues the MMAs, w 5.. (NPROD warps)
// produce.  Producers read `in` from global memory in its own storage order
// with whole-line warp accesses (a float4 of four adjacent columns per lane
// at one direction when a column axis is fastest, 512 contiguous bytes per
// warp; a column's 128-byte run of 32 directions per eight lanes when d is
// fastest), split each value into tf32 hi/lo and write both into a
// STAGES-deep ring of K-major operand tiles (128 columns x 32 directions, no
// swizzle: 8x16-byte core matrices, K-adjacent ones LBO = 144 B apart, 8-row
// groups SBO = 1168 B apart; the 16-byte pads make both write patterns
// conflict-free).  L's hi/lo parts are laid out once per block with LBO =
// 128 B and SBO = DP*32 B.  Two accumulators of NPA
// columns let the epilogue of one tile overlap the MMAs of the next.
//
// AT = 1 (mode 6) keeps the A operand in tensor memory instead: converter
// warp w reads its tile rows (TMEM lanes 32 (w % 4) ..) from the TMA box,
// splits them and writes tf32 hi and lo with tcgen05.st into a STAGES-deep
// ring of TMEM stages (32 hi + 32 lo columns each, after the accumulators);
// the MMAs read A from tensor memory and only B (L) from shared memory.  Per
// 4-byte element of `in` shared memory then carries the TMA write and one
// converter read (8 bytes) instead of those plus the operand writes and the
// three MMAs' A reads (28 bytes), the traffic that bounds the shared-memory
// form.  Every
// wait is bounded (about a second): on expiry the block raises its abort
// flag, counts the event in cj_wait_timeouts, drains its MMAs, frees TMEM
// and returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lt_smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void lt_mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void lt_mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool lt_mbar_test(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long lt_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` to complete; false after about a
// second, or at once when abort_flag (if given) is up.
__device__ __forceinline__ bool lt_mbar_wait(unsigned bar, unsigned parity, volatile int* abort_flag) {
    if (lt_mbar_test(bar, parity)) return true;
    const unsigned long long t0 = lt_globaltimer();
    for (;;) {
        if (lt_mbar_test(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (lt_globaltimer() - t0 > 1000000000ull) return false;
    }
}
__device__ __forceinline__ void lt_tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void lt_tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void lt_tc_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// Shared-memory matrix descriptor, K-major without swizzle: start address,
// leading byte offset (K-adjacent core matrices), stride byte offset (8-row
// groups), descriptor version 1 at bit 46, swizzle mode 0.
__device__ __forceinline__ unsigned long long lt_tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void lt_tc_mma_tf32(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                               unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The same with A read from tensor memory (a_tmem: lane 0, the first of the
// 8 columns that hold this K step's tf32 elements); B from shared memory.
__device__ __forceinline__ void lt_tc_mma_tf32_ts(unsigned d_tmem, unsigned a_tmem, unsigned long long b,
                                                  unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// A TMA tensor map (the driver's 128-byte CUtensorMap), passed by value as a
// __grid_constant__ kernel parameter.
struct alignas(64) cj_tmap {
    unsigned long long v[16];
};
__device__ __forceinline__ void lt_mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One box of a 3-D tensor map (coordinates innermost first) into shared
// memory; completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void lt_tma_load_3d(unsigned dst, const cj_tmap* map, int c0, int c1, int c2, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
// Columns c..c+15 of this thread's TMEM lane (warp w reads lanes 32(w%4)..).
__device__ __forceinline__ void lt_tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    // the registers are valid only after wait::ld; passing them through it
    // keeps every use behind the wait
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Columns c..c+15 of this thread's TMEM lane from registers (warp w writes
// lanes 32(w%4)..); complete once tcgen05.wait::st returns.
__device__ __forceinline__ void lt_tmem_st16(unsigned taddr, const unsigned (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// Store the staged out box of one tile (see ltimes_tc): units of V
// consecutive elements along out's faster column axis A2 (1 = g, 2 = z),
// walked in out's storage order by the 128 epilogue threads.  Box layout:
// box[m * OUTER * RUNP + outer * RUNP + inner].
template <int V, int M, int A2, int RUN, int OUTER, int RUNP, bool M_SLOWEST, int ACC>
__device__ __forceinline__ void lt_tc_store_box(float* __restrict__ out, const float* box, long long G, long long Z,
                                                long long g0, long long z0, const long long (&so)[3], int r) {
    constexpr int NV = RUN / V, UNITS = M * OUTER * NV, MS = OUTER * RUNP;
    for (int u = r; u < UNITS; u += 128) {
        const int iv = u % NV, rest = u / NV;
        const int o = M_SLOWEST ? rest % OUTER : rest / M;
        const int m = M_SLOWEST ? rest / OUTER : rest % M;
        const int inner = iv * V;
        const long long g = g0 + (A2 == 1 ? inner : o), z = z0 + (A2 == 1 ? o : inner);
        if (g >= G || z >= Z) continue;
        float* p = out + m * so[0] + g * so[1] + z * so[2];
        const float* q = box + m * MS + o * RUNP + inner;
        if constexpr (V == 4) {
            float4 x = *reinterpret_cast<const float4*>(q);
            if (ACC) {
                const float4 w = *reinterpret_cast<const float4*>(p);
                x.x += w.x; x.y += w.y; x.z += w.z; x.w += w.w;
            }
            *reinterpret_cast<float4*>(p) = x;
        } else {
            *p = ACC ? *p + *q : *q;
        }
    }
}

// Same for out with m fastest: box[column * MP + m], columns in out's order
// (outer column axis slower, A1 the faster one with extent RIN); units of V
// consecutive moments.
template <int V, int M, int A1, int RIN, int MP, int ACC>
__device__ __forceinline__ void lt_tc_store_mbox(float* __restrict__ out, const float* box, long long G, long long Z,
                                                 long long g0, long long z0, const long long (&so)[3], int r) {
    constexpr int NV = M / V, UNITS = 128 * NV;
    for (int u = r; u < UNITS; u += 128) {
        const int mv = u % NV, ci = u / NV;
        const int inner = ci % RIN, outer = ci / RIN;
        const long long g = g0 + (A1 == 1 ? inner : outer), z = z0 + (A1 == 1 ? outer : inner);
        if (g >= G || z >= Z) continue;
        float* p = out + g * so[1] + z * so[2] + mv * V;
        const float* q = box + ci * MP + mv * V;
        if constexpr (V == 4) {
            float4 x = *reinterpret_cast<const float4*>(q);
            if (ACC) {
                const float4 w = *reinterpret_cast<const float4*>(p);
                x.x += w.x; x.y += w.y; x.z += w.z; x.w += w.w;
            }
            *reinterpret_cast<float4*>(p) = x;
        } else {
            *p = ACC ? *p + *q : *q;
        }
    }
}

template <int M, int D, int LIN, int LOUT, int TG, int TZ, int STAGES, int NPROD, int PF_ = 0, int RAWST = 0,
          int ACC = 0, int INJECT_TIMEOUT = 0, int AT = 0>
__global__ void __maxnreg__(cjg::lt_tc_maxreg(NPROD + (RAWST > 0)))
ltimes_tc(const float* __restrict__ L, const float* __restrict__ in, float* __restrict__ out, long long G, long long Z,
          const __grid_constant__ cj_tmap tmap) {
    constexpr int BM = 128, KB = 32;                 // tile columns, directions per stage
    constexpr int NP = cjg::lt_tc_np(M), DP = cjg::lt_tc_dp(D), NKB = DP / KB;
    constexpr int NPA = (NP + 31) / 32 * 32;         // TMEM columns per accumulator
    constexpr int ACOLS = AT ? STAGES * 2 * KB : 0;   // TMEM operand stages (AT): hi and lo, after the accumulators
    constexpr int TUSE = 2 * NPA + ACOLS;
    constexpr int TCOLS = TUSE <= 32 ? 32 : TUSE <= 64 ? 64 : TUSE <= 128 ? 128 : TUSE <= 256 ? 256 : 512;
    constexpr int PT = 32 * NPROD;                   // producer (converter) threads
    constexpr int PW0 = RAWST > 0 ? 6 : 5;           // first producer warp (warp 5 issues TMA in mode 5)
    constexpr unsigned RAW_BYTES = BM * KB * 4u;     // one TMA box of `in`
    constexpr int CH = BM * KB / 4 / PT;             // 16-byte chunks per producer thread per stage
    constexpr unsigned A_LBO = cjg::LT_TC_A_LBO, A_SBO = cjg::LT_TC_A_SBO;
    constexpr unsigned HALF = cjg::LT_TC_A_BYTES, STAGE_BYTES = 2u * HALF;
    constexpr unsigned LBYTES = NP * DP * 4u;
    constexpr unsigned B_SBO = (DP / 4) * 128u;
    // kind::tf32, FP32 accumulator, both operands K-major, N = NP, M = 128
    constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NP >> 3) << 17) | ((128u >> 4) << 24);
    // register producers split the 8 direction quads of a stage over warps; converters only need whole chunks
    static_assert(TG * TZ == BM && NP <= 256 && CH * PT * 4 == BM * KB && (RAWST > 0 ? 32 : 8) % NPROD == 0,
                  "tcgen05 LTimes tile");
    // TMEM operands: fed by TMA, each lane quarter's warps split a stage's directions, all stages fit TMEM
    static_assert(!AT || (RAWST > 0 && NPROD % 4 == 0 && KB % (NPROD / 4 * 8) == 0 && TUSE <= 512),
                  "tcgen05 LTimes tile with tensor-memory operands");
    // a TMA box starts on a 16-byte boundary: its innermost extent (and so
    // every innermost coordinate, a multiple of it) is a multiple of 4 floats
    static_assert(RAWST == 0 || (lt_axis(LIN, 2) == 0 ? KB : lt_axis(LIN, 2) == 1 ? TG : TZ) % 4 == 0,
                  "TMA box: innermost extent must be a multiple of 4");
    constexpr bool G_FASTER = lt_pos(LIN, 1) > lt_pos(LIN, 2);
    constexpr bool OUT_G_FASTER = lt_pos(LOUT, 1) > lt_pos(LOUT, 2);
    constexpr bool D_FAST = lt_pos(LIN, 0) == 2;
    constexpr bool M_FAST = lt_pos(LOUT, 0) == 2;
    // Each thread stores its own tile row straight from registers when out
    // has a column axis fastest and orders its column axes like in (a warp
    // then writes 128 contiguous bytes per moment).  Otherwise the tile goes
    // through a staged box in shared memory and is stored in out's order as
    // float4 units:
    //  * column axis fastest in out: runs along that axis (RUN floats, padded
    //    to RUNP so the TMEM -> box writes spread over all banks), box index
    //    m * MS + outer * RUNP + inner;
    //  * m fastest in out: one row of MP floats per column, columns in out's
    //    order (MP / 4 odd: conflict-free 16-byte writes), box index
    //    column * MP + m.
    constexpr bool DIRECT_OUT = !M_FAST && G_FASTER == OUT_G_FASTER;
    constexpr int A2 = lt_axis(LOUT, 2);                  // 1 = g, 2 = z, 0 = m
    constexpr int RUN = A2 == 1 ? TG : TZ, OUTER = BM / RUN;
    constexpr int RUNP = cjg::lt_tc_runp(RUN), MS = OUTER * RUNP;
    constexpr bool M_SLOWEST = lt_pos(LOUT, 0) == 0;
    constexpr int A1 = lt_axis(LOUT, 1);                  // m fastest: out's faster column axis
    constexpr int RIN = A1 == 1 ? TG : TZ, MP = cjg::lt_tc_mp(M);

    extern __shared__ __align__(16) unsigned char cj_smem[];
    __shared__ __align__(8) unsigned long long bars[2 * STAGES + 6 + 2 * RAWST];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    unsigned char* base = cj_smem + ((1024u - (lt_smem_u32(cj_smem) & 1023u)) & 1023u);
    unsigned char* raw = base;                                    // RAWST TMA boxes (mode 5)
    unsigned char* ring = base + RAWST * RAW_BYTES;               // STAGES x [A_hi | A_lo]
    constexpr unsigned RING_BYTES = AT ? 0u : STAGES * STAGE_BYTES;   // the operand ring is in TMEM when AT
    float* sLhi = reinterpret_cast<float*>(ring + RING_BYTES);
    float* sLlo = reinterpret_cast<float*>(ring + RING_BYTES + LBYTES);
    float* sO = reinterpret_cast<float*>(ring + RING_BYTES + 2 * LBYTES);
    const unsigned ring_u = lt_smem_u32(ring), lhi_u = lt_smem_u32(sLhi), llo_u = lt_smem_u32(sLlo);
    const unsigned bar_u = lt_smem_u32(bars);
    auto full_bar = [&](int s) { return bar_u + 8u * s; };
    auto empty_bar = [&](int s) { return bar_u + 8u * (STAGES + s); };
    auto accf_bar = [&](int a) { return bar_u + 8u * (2 * STAGES + a); };
    auto acce_bar = [&](int a) { return bar_u + 8u * (2 * STAGES + 2 + a); };
    const unsigned done_bar = bar_u + 8u * (2 * STAGES + 4);
    const unsigned epi_bar = bar_u + 8u * (2 * STAGES + 5);   // the 128 epilogue threads
    auto rawf_bar = [&](int s) { return bar_u + 8u * (2 * STAGES + 6 + s); };
    auto rawe_bar = [&](int s) { return bar_u + 8u * (2 * STAGES + 6 + RAWST + s); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            lt_mbar_init(full_bar(s), PT);
            lt_mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            lt_mbar_init(accf_bar(a), 1);
            lt_mbar_init(acce_bar(a), 4 * 32);
        }
        lt_mbar_init(done_bar, 1);
        lt_mbar_init(epi_bar, 4 * 32);
        for (int s = 0; s < RAWST; ++s) {
            lt_mbar_init(rawf_bar(s), 1);
            lt_mbar_init(rawe_bar(s), PT);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(lt_smem_u32(&tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // L (hi and lo) in the K-major core-matrix layout, zero-padded to NP x DP
    for (int e = tid; e < NP * DP; e += blockDim.x) {
        const int n = e / DP, k = e - n * DP;
        const float v = (n < M && k < D) ? L[n * D + k] : 0.f;
        const unsigned hi = to_tf32(v);
        const unsigned off = (k >> 2) * 128u + (n >> 3) * B_SBO + (n & 7) * 16u + (k & 3) * 4u;
        reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(sLhi) + off)[0] = hi;
        reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(sLlo) + off)[0] = to_tf32(v - __uint_as_float(hi));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    lt_tc_fence_before();
    __syncthreads();
    lt_tc_fence_after();
    const unsigned tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;
    auto give_up = [&]() {
        if (atomicExch(&abort_flag, 1) == 0) atomicAdd(&cj_wait_timeouts, 1u);
    };

    const long long ext[3] = {D, G, Z};
    long long st[3], so[3];
    st[lt_axis(LIN, 2)] = 1;
    st[lt_axis(LIN, 1)] = ext[lt_axis(LIN, 2)];
    st[lt_axis(LIN, 0)] = ext[lt_axis(LIN, 2)] * ext[lt_axis(LIN, 1)];
    const long long exo[3] = {M, G, Z};
    so[lt_axis(LOUT, 2)] = 1;
    so[lt_axis(LOUT, 1)] = exo[lt_axis(LOUT, 2)];
    so[lt_axis(LOUT, 0)] = exo[lt_axis(LOUT, 2)] * exo[lt_axis(LOUT, 1)];
    // Tile t covers g-block t % ntg and z-block t / ntg: the tiles that share
    // a z range (and so the cache lines of a g-fastest tensor) run at the
    // same time on neighbouring blocks and meet in L2.
    const long long ntg = (G + TG - 1) / TG;
    const long long ntiles = ntg * ((Z + TZ - 1) / TZ);
    const unsigned ntg32 = (unsigned)ntg;
    // tile row r (0..127) -> (gl, zl), rows in the order of in's faster column axis
    auto row_g = [&](int r) { return G_FASTER ? r % TG : r / TZ; };
    auto row_z = [&](int r) { return G_FASTER ? r / TG : r % TZ; };

    const long long n_it = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x * NKB;   // this block's stages
    if (AT && warp >= PW0) {
        if constexpr (AT) {
            // ---------------- converters, TMEM operands (mode 6) ----------------
            // Warp w owns tile rows (TMEM lanes) 32 (w % 4) + lane; the NPROD / 4
            // warps of one lane quarter take KP consecutive directions of each
            // raw box.  d fastest: 16-byte chunks of the row's 128-byte swizzled
            // run; otherwise one float per direction, consecutive rows across the
            // warp.  Each value is split into tf32 hi/lo and both go to TMEM
            // stage s with tcgen05.st (hi in its first KB columns, lo in the next).
            constexpr int KP = KB / (NPROD / 4);
            constexpr int AI = lt_axis(LIN, 2), AM = lt_axis(LIN, 1);
            constexpr int BI = AI == 0 ? KB : AI == 1 ? TG : TZ, BMID = AM == 0 ? KB : AM == 1 ? TG : TZ;
            constexpr int SB0 = AI == 0 ? 1 : AM == 0 ? BI : BI * BMID;   // raw element strides of d, g, z
            constexpr int SB1 = AI == 1 ? 1 : AM == 1 ? BI : BI * BMID;
            constexpr int SB2 = AI == 2 ? 1 : AM == 2 ? BI : BI * BMID;
            const int quarter = warp & 3, part = (warp - PW0) >> 2;
            const int r = 32 * quarter + lane;
            const unsigned trow = tmem + ((unsigned)(32 * quarter) << 16) + 2 * NPA + part * KP;
            const int roff = D_FAST ? 0 : row_g(r) * SB1 + row_z(r) * SB2;
            for (long long i = 0; i < n_it; ++i) {
                const int rs = (int)(i % RAWST), s = (int)(i % STAGES);
                if (!lt_mbar_wait(rawf_bar(rs), (unsigned)((i / RAWST) & 1), abort_v) ||
                    !lt_mbar_wait(empty_bar(s), (unsigned)((i / STAGES) & 1) ^ 1u, abort_v)) {
                    give_up();
                    break;
                }
                lt_tc_fence_after();
                const unsigned char* rb = raw + rs * RAW_BYTES;
                float x[KP];
                if constexpr (D_FAST) {
#pragma unroll
                    for (int c = 0; c < KP / 4; ++c) {
                        const int kq = part * (KP / 4) + c;
                        const float4 v = *reinterpret_cast<const float4*>(rb + r * 128 + ((kq ^ (r & 7)) << 4));
                        x[4 * c] = v.x;
                        x[4 * c + 1] = v.y;
                        x[4 * c + 2] = v.z;
                        x[4 * c + 3] = v.w;
                    }
                } else {
                    const float* rf = reinterpret_cast<const float*>(rb) + roff;
#pragma unroll
                    for (int j = 0; j < KP; ++j) x[j] = rf[(part * KP + j) * SB0];
                }
                lt_mbar_arrive(rawe_bar(rs));   // the box is read: the TMA lane may refill it
                const unsigned ts = trow + (unsigned)(s * 2 * KB);
#pragma unroll
                for (int h = 0; h < KP; h += 16) {
                    unsigned vh[16], vl[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        vh[j] = to_tf32(x[h + j]);
                        vl[j] = to_tf32(x[h + j] - __uint_as_float(vh[j]));
                    }
                    lt_tmem_st16(ts + h, vh);
                    lt_tmem_st16(ts + KB + h, vl);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                lt_tc_fence_before();
                if (!INJECT_TIMEOUT) lt_mbar_arrive(full_bar(s));   // the hook: never signal a filled stage
            }
        }
    } else if (RAWST > 0 && warp >= PW0) {
        // ---------------- converters (mode 5) ----------------
        // Raw box i (in's storage order; 128-byte swizzled rows when d is
        // fastest) -> tf32 hi/lo K-major operand stage.  d fastest: chunk q is
        // (row q >> 3, direction quad q & 7), one 16-byte read; otherwise
        // chunk q is (row q & 127, quad q >> 7), four 4-byte reads at
        // consecutive rows across the warp.
        constexpr int RS = RAWST > 0 ? RAWST : 1;
        constexpr int AI = lt_axis(LIN, 2), AM = lt_axis(LIN, 1);
        constexpr int BI = AI == 0 ? KB : AI == 1 ? TG : TZ, BMID = AM == 0 ? KB : AM == 1 ? TG : TZ;
        constexpr int SB0 = AI == 0 ? 1 : AM == 0 ? BI : BI * BMID;   // raw element strides of d, g, z
        constexpr int SB1 = AI == 1 ? 1 : AM == 1 ? BI : BI * BMID;
        constexpr int SB2 = AI == 2 ? 1 : AM == 2 ? BI : BI * BMID;
        const int pt = tid - PW0 * 32;
        for (long long i = 0; i < n_it; ++i) {
            const int rs = (int)(i % RS), s = (int)(i % STAGES);
            if (!lt_mbar_wait(rawf_bar(rs), (unsigned)((i / RS) & 1), abort_v) ||
                !lt_mbar_wait(empty_bar(s), (unsigned)((i / STAGES) & 1) ^ 1u, abort_v)) {
                give_up();
                break;
            }
            const unsigned char* rb = raw + rs * RAW_BYTES;
            unsigned char* hi = ring + s * STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int q = j * PT + pt;
                float4 c;
                int r, kq;
                if constexpr (D_FAST) {
                    r = q >> 3;
                    kq = q & 7;
                    c = *reinterpret_cast<const float4*>(rb + r * 128 + ((kq ^ (r & 7)) << 4));
                } else {
                    r = q & 127;
                    kq = q >> 7;
                    const float* rf = reinterpret_cast<const float*>(rb) + row_g(r) * SB1 + row_z(r) * SB2;
                    c = make_float4(rf[(4 * kq) * SB0], rf[(4 * kq + 1) * SB0], rf[(4 * kq + 2) * SB0],
                                    rf[(4 * kq + 3) * SB0]);
                }
                uint4 h, l;
                h.x = to_tf32(c.x); l.x = to_tf32(c.x - __uint_as_float(h.x));
                h.y = to_tf32(c.y); l.y = to_tf32(c.y - __uint_as_float(h.y));
                h.z = to_tf32(c.z); l.z = to_tf32(c.z - __uint_as_float(h.z));
                h.w = to_tf32(c.w); l.w = to_tf32(c.w - __uint_as_float(h.w));
                const unsigned off = kq * A_LBO + (r >> 3) * A_SBO + (r & 7) * 16u;
                *reinterpret_cast<uint4*>(hi + off) = h;
                *reinterpret_cast<uint4*>(hi + HALF + off) = l;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (!INJECT_TIMEOUT) lt_mbar_arrive(full_bar(s));   // the hook: never signal a filled stage
            lt_mbar_arrive(rawe_bar(rs));
        }
    } else if (RAWST > 0 && warp == 5) {
        // ---------------- TMA issue (mode 5, one lane) ----------------
        if (lane == 0) {
            constexpr int RS = RAWST > 0 ? RAWST : 1;
            long long issued = 0;
            for (long long i = 0; i < n_it; ++i, ++issued) {
                const int rs = (int)(i % RS);
                if (!lt_mbar_wait(rawe_bar(rs), (unsigned)((i / RS) & 1) ^ 1u, abort_v)) {
                    give_up();
                    break;
                }
                const unsigned t = blockIdx.x + (unsigned)(i / NKB) * gridDim.x;
                const int c[3] = {(int)(i % NKB) * KB, (int)(t % ntg32) * TG, (int)(t / ntg32) * TZ};   // d, g, z
                lt_mbar_expect_tx(rawf_bar(rs), RAW_BYTES);
                lt_tma_load_3d(lt_smem_u32(raw + rs * RAW_BYTES), &tmap, c[lt_axis(LIN, 2)], c[lt_axis(LIN, 1)],
                               c[lt_axis(LIN, 0)], rawf_bar(rs));
            }
            // every issued box lands before the block can exit: wait (bounded,
            // not cut short by the abort flag) for the last load into each slot
            for (int s = 0; s < RS; ++s) {
                const long long cnt = issued > s ? (issued - s + RS - 1) / RS : 0;
                if (cnt > 0 && !lt_mbar_wait(rawf_bar(s), (unsigned)((cnt - 1) & 1), nullptr)) give_up();
            }
        }
        __syncwarp();
    } else if (RAWST == 0 && warp >= PW0) {
        // ---------------- producers ----------------
        // Iteration i of this block is tile blockIdx.x + (i / NKB) * gridDim.x,
        // K block i % NKB.  Loads run PF - 1 iterations ahead in a register
        // ring of PF * CH float4 (PF_ = 0: what the register cap leaves), so
        // several stages of `in` are in flight per thread while it waits for
        // a free operand stage.  Tile indices fit 32 bits (G * Z < 2^38).
        constexpr int PF_AUTO = (cjg::lt_tc_maxreg(NPROD) - 64) / (4 * CH);
        constexpr int PF = PF_ > 0 ? PF_ : (PF_AUTO < 1 ? 1 : PF_AUTO > 8 ? 8 : PF_AUTO);
        const int pt = tid - PW0 * 32;
        // Column-fastest `in`: warp wp loads direction quads kq = wp * UPW ..
        // (UPW = 8 / NPROD), lane l columns 4l..4l+3 (a float4 when the
        // fastest column axis has a multiple-of-4 extent, else scalars);
        // v[4 * uu + dd] holds direction 4 kq + dd.  d-fastest `in`: chunk q
        // of the stage is (row q >> 3, quad q & 7), a float4 along d.
        constexpr int UPW = 8 / NPROD > 0 ? 8 / NPROD : 1;
        const int wp = pt >> 5, c0 = 4 * (pt & 31);
        const long long fast_ext = G_FASTER ? G : Z;
        const bool vec4 = D_FAST ? (D % 4 == 0) : (fast_ext % 4 == 0 && (G_FASTER ? TG : TZ) % 4 == 0);
        auto load = [&](long long i, float4 (&v)[CH]) {
            const unsigned t = blockIdx.x + (unsigned)(i / NKB) * gridDim.x;
            const int kb = (int)(i % NKB);
            const long long g0 = (long long)(t % ntg32) * TG, z0 = (long long)(t / ntg32) * TZ;
            if constexpr (D_FAST) {
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int q = j * PT + pt;
                    const int r = q >> 3, d0 = kb * KB + (q & 7) * 4;
                    const long long g = g0 + row_g(r), z = z0 + row_z(r);
                    const bool ok = g < G && z < Z;
                    const float* p = in + (ok ? g * st[1] + z * st[2] : 0);
                    if (vec4) {
                        v[j] = (ok && d0 < D) ? __ldg(reinterpret_cast<const float4*>(p + d0))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        v[j].x = (ok && d0 + 0 < D) ? __ldg(p + d0 + 0) : 0.f;
                        v[j].y = (ok && d0 + 1 < D) ? __ldg(p + d0 + 1) : 0.f;
                        v[j].z = (ok && d0 + 2 < D) ? __ldg(p + d0 + 2) : 0.f;
                        v[j].w = (ok && d0 + 3 < D) ? __ldg(p + d0 + 3) : 0.f;
                    }
                }
            } else {
                const long long g = g0 + row_g(c0), z = z0 + row_z(c0);   // first of the four columns
                const long long cbase = g * st[1] + z * st[2];
#pragma unroll
                for (int uu = 0; uu < UPW; ++uu)
#pragma unroll
                    for (int dd = 0; dd < 4; ++dd) {
                        const int d = kb * KB + (wp * UPW + uu) * 4 + dd;
                        float4& x = v[4 * uu + dd];
                        if (vec4) {
                            x = (g < G && z < Z && d < D)
                                    ? __ldg(reinterpret_cast<const float4*>(in + cbase + (long long)d * st[0]))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                        } else {
                            float e[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const long long gc = g0 + row_g(c0 + c), zc = z0 + row_z(c0 + c);
                                e[c] = (gc < G && zc < Z && d < D)
                                           ? __ldg(in + gc * st[1] + zc * st[2] + (long long)d * st[0])
                                           : 0.f;
                            }
                            x = make_float4(e[0], e[1], e[2], e[3]);
                        }
                    }
            }
        };
        float4 buf[PF][CH];
#pragma unroll
        for (int u = 0; u < PF - 1; ++u)
            if (u < n_it) load(u, buf[u]);
        bool live = true;
        for (long long i0 = 0; live && i0 < n_it; i0 += PF) {
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const long long i = i0 + u;
                if (i >= n_it) break;
                if (i + PF - 1 < n_it) load(i + PF - 1, buf[(u + PF - 1) % PF]);
                const int s = (int)(i % STAGES);
                if (!lt_mbar_wait(empty_bar(s), (unsigned)((i / STAGES) & 1) ^ 1u, abort_v)) {
                    give_up();
                    live = false;
                    break;
                }
                unsigned char* hi = ring + s * STAGE_BYTES;
                auto put = [&](unsigned off, float4 c) {   // one 16-byte row of a core matrix, hi and lo
                    uint4 h, l;
                    h.x = to_tf32(c.x); l.x = to_tf32(c.x - __uint_as_float(h.x));
                    h.y = to_tf32(c.y); l.y = to_tf32(c.y - __uint_as_float(h.y));
                    h.z = to_tf32(c.z); l.z = to_tf32(c.z - __uint_as_float(h.z));
                    h.w = to_tf32(c.w); l.w = to_tf32(c.w - __uint_as_float(h.w));
                    *reinterpret_cast<uint4*>(hi + off) = h;
                    *reinterpret_cast<uint4*>(hi + HALF + off) = l;
                };
                if constexpr (D_FAST) {
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int q = j * PT + pt, r = q >> 3;
                        put((q & 7) * A_LBO + (r >> 3) * A_SBO + (r & 7) * 16u, buf[u][j]);
                    }
                } else {
                    // 4 x 4 transpose in registers: column c0 + c, directions 4 kq .. 4 kq + 3
#pragma unroll
                    for (int uu = 0; uu < UPW; ++uu)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float4* w = &buf[u][4 * uu];
                            const float4 col = c == 0 ? make_float4(w[0].x, w[1].x, w[2].x, w[3].x)
                                             : c == 1 ? make_float4(w[0].y, w[1].y, w[2].y, w[3].y)
                                             : c == 2 ? make_float4(w[0].z, w[1].z, w[2].z, w[3].z)
                                                      : make_float4(w[0].w, w[1].w, w[2].w, w[3].w);
                            const int r = c0 + c;
                            put((wp * UPW + uu) * A_LBO + (r >> 3) * A_SBO + (r & 7) * 16u, col);
                        }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (!INJECT_TIMEOUT) lt_mbar_arrive(full_bar(s));
            }
        }
    } else if (warp == 4) {
        // ---------------- MMA issue (one lane) ----------------
        if (lane == 0) {
            int it = 0, tl = 0;
            bool ok = true;
            for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++tl) {
                const int a = tl & 1;
                if (!lt_mbar_wait(acce_bar(a), ((tl >> 1) & 1) ^ 1, abort_v)) {
                    give_up();
                    break;
                }
                lt_tc_fence_after();
                const unsigned dt = tmem + a * NPA;
                for (int kb = 0; kb < NKB; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!lt_mbar_wait(full_bar(s), (it / STAGES) & 1, abort_v)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    lt_tc_fence_after();
                    if constexpr (AT) {
                        const unsigned acol = tmem + 2 * NPA + (unsigned)(s * 2 * KB);   // hi; lo KB columns on
#pragma unroll
                        for (int j = 0; j < KB / 8; ++j) {
                            const unsigned bo = (kb * (KB / 4) + 2 * j) * 128u;
                            const unsigned long long dbh = lt_tc_desc(lhi_u + bo, 128u, B_SBO);
                            const unsigned long long dbl = lt_tc_desc(llo_u + bo, 128u, B_SBO);
                            lt_tc_mma_tf32_ts(dt, acol + KB + 8 * j, dbh, IDESC, (kb | j) != 0);
                            lt_tc_mma_tf32_ts(dt, acol + 8 * j, dbl, IDESC, 1u);
                            lt_tc_mma_tf32_ts(dt, acol + 8 * j, dbh, IDESC, 1u);
                        }
                        lt_tc_commit(empty_bar(s));   // the TMEM stage is free once these MMAs have read it
                        continue;
                    }
                    const unsigned ahi = ring_u + s * STAGE_BYTES, alo = ahi + HALF;
#pragma unroll
                    for (int j = 0; j < KB / 8; ++j) {
                        const unsigned bo = (kb * (KB / 4) + 2 * j) * 128u;
                        const unsigned long long dah = lt_tc_desc(ahi + 2 * j * A_LBO, A_LBO, A_SBO);
                        const unsigned long long dal = lt_tc_desc(alo + 2 * j * A_LBO, A_LBO, A_SBO);
                        const unsigned long long dbh = lt_tc_desc(lhi_u + bo, 128u, B_SBO);
                        const unsigned long long dbl = lt_tc_desc(llo_u + bo, 128u, B_SBO);
                        lt_tc_mma_tf32(dt, dal, dbh, IDESC, (kb | j) != 0);
                        lt_tc_mma_tf32(dt, dah, dbl, IDESC, 1u);
                        lt_tc_mma_tf32(dt, dah, dbh, IDESC, 1u);
                    }
                    lt_tc_commit(empty_bar(s));   // the stage is free once these MMAs have read it
                }
                if (!ok) break;
                lt_tc_commit(accf_bar(a));
            }
            // drain: every MMA issued above completes before TMEM is freed
            // (bounded, and not cut short by the abort flag)
            lt_tc_commit(done_bar);
            if (!lt_mbar_wait(done_bar, 0, nullptr)) give_up();
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-3: tile rows 32w..32w+31) ----------------
        const int r = tid;   // TMEM lane = tile row
        int tl = 0, epi_use = 0;
        // all 128 epilogue threads meet (bounded; an mbarrier, so that a
        // thread that gives up cannot leave the others blocked)
        auto epi_sync = [&]() {
            lt_mbar_arrive(epi_bar);
            const bool met = lt_mbar_wait(epi_bar, epi_use & 1, abort_v);
            ++epi_use;
            return met;
        };
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const int a = tl & 1;
            if (!lt_mbar_wait(accf_bar(a), (tl >> 1) & 1, abort_v)) {
                give_up();
                break;
            }
            lt_tc_fence_after();
            const long long g0 = (t % ntg) * TG, z0 = (t / ntg) * TZ;
            const int gl = row_g(r), zl = row_z(r);
            const bool ok = g0 + gl < G && z0 + zl < Z;
            float* o = out + (ok ? (g0 + gl) * so[1] + (z0 + zl) * so[2] : 0);
            if constexpr (!DIRECT_OUT) {
                if (!epi_sync()) {   // the previous box has been stored
                    give_up();
                    break;
                }
            }
            // 16 accumulator columns (moments) at a time: TMEM -> registers -> out or the box
#pragma unroll
            for (int c = 0; c < NP; c += 16) {
                float v[16];
                lt_tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + a * NPA + c, v);
                if constexpr (DIRECT_OUT) {
                    if (ok) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            if (c + i >= M) break;
                            float* pp = o + (c + i) * so[0];
                            *pp = ACC ? *pp + v[i] : v[i];
                        }
                    }
                } else if constexpr (M_FAST) {
                    const int ci = (A1 == 1 ? zl : gl) * RIN + (A1 == 1 ? gl : zl);   // column in out's order
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4)
                        if (c + 4 * i4 < MP)
                            *reinterpret_cast<float4*>(sO + ci * MP + c + 4 * i4) =
                                make_float4(v[4 * i4], v[4 * i4 + 1], v[4 * i4 + 2], v[4 * i4 + 3]);
                } else {
                    const int oidx = (A2 == 1 ? zl : gl) * RUNP + (A2 == 1 ? gl : zl);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c + i < M) sO[(c + i) * MS + oidx] = v[i];
                }
            }
            lt_tc_fence_before();
            lt_mbar_arrive(acce_bar(a));   // the accumulator may be overwritten
            if constexpr (!DIRECT_OUT) {
                if (!epi_sync()) {
                    give_up();
                    break;
                }
                if constexpr (M_FAST) {
                    if (M % 4 == 0)
                        lt_tc_store_mbox<(M % 4 == 0 ? 4 : 1), M, A1, RIN, MP, ACC>(out, sO, G, Z, g0, z0, so, r);
                    else
                        lt_tc_store_mbox<1, M, A1, RIN, MP, ACC>(out, sO, G, Z, g0, z0, so, r);
                } else if (RUN % 4 == 0 && (A2 == 1 ? G : Z) % 4 == 0)
                    lt_tc_store_box<(RUN % 4 == 0 ? 4 : 1), M, A2, RUN, OUTER, RUNP, M_SLOWEST, ACC>(out, sO, G, Z, g0, z0,
                                                                                                  so, r);
                else
                    lt_tc_store_box<1, M, A2, RUN, OUTER, RUNP, M_SLOWEST, ACC>(out, sO, G, Z, g0, z0, so, r);
            }
        }
    }
    lt_tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        lt_tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// Generic: run-time M, D, strides and accumulate flag; one thread per column q = g*Z + z
// (z fastest), blockDim.x columns per block.  The column's D inputs are
// staged in shared memory with the thread's own loads (coalesced only when z
// is the fastest axis of `in`), L is read from shared memory.
template <class T>
__global__ void __launch_bounds__(128)
ltimes_generic(const T* __restrict__ L, const T* __restrict__ in, T* __restrict__ out, long long G,
               long long Z, int M, int D, long long si_x, long long si_g, long long si_z,
               long long so_x, long long so_g, long long so_z, int acc) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sL = reinterpret_cast<T*>(cj_smem);
    const int cols = blockDim.x;
    T* sX = sL + M * D;
    const int tid = threadIdx.x;
    for (int e = tid; e < M * D; e += cols) sL[e] = L[e];
    const long long q = (long long)blockIdx.x * cols + tid;
    const bool ok = q < G * Z;
    const long long g = ok ? q / Z : 0, z = ok ? q - (q / Z) * Z : 0;
    if (ok)
        for (int d = 0; d < D; ++d) sX[d * cols + tid] = in[d * si_x + g * si_g + z * si_z];
    __syncthreads();
    if (!ok) return;
    for (int m = 0; m < M; ++m) {
        T s = T(0);
        for (int d = 0; d < D; ++d) s = lt_fma(sL[m * D + d], sX[d * cols + tid], s);
        T* o = out + m * so_x + g * so_g + z * so_z;
        *o = acc ? *o + s : s;
    }
}

}  // namespace cj
#endif
