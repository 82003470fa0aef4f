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
