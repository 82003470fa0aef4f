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
template <class T, int LAY, int EX, int TG, int TZ, int CP, int NT, bool LOAD>
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
        else if (ok) g[goff] = *sp;
    }
}

// Persistent kernel: L^T stays in shared memory; each block loops over
// (g, z) tiles: stage the in box, contract, stage and store the out box.
template <class T, int M, int D, int LIN, int LOUT, int TG, int TZ, int NT, int R, int S>
__global__ void __launch_bounds__(NT)
ltimes(const T* __restrict__ L, const T* __restrict__ in, T* __restrict__ out, long long G, long long Z) {
    constexpr int CT = TG * TZ;
    constexpr int MG = (M + S - 1) / S;   // moment groups (the last may be partial)
    constexpr int MP = cjg::lt_mpitch(MG * S, (int)sizeof(T));
    constexpr int CP = cjg::lt_cpitch(CT, (int)sizeof(T));
    constexpr int QG = CT / R;   // column groups
    static_assert(CT % R == 0 && QG * MG == NT, "tile does not cover the block");
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sL = reinterpret_cast<T*>(cj_smem);   // [D][MP], L transposed
    T* sX = sL + D * MP;                      // [D][CP] in tile, then [M][CP] out tile
    const int tid = threadIdx.x;
    for (int e = tid; e < MP * D; e += NT) {
        const int m = e / D, d = e - m * D;
        sL[d * MP + m] = m < M ? L[e] : T(0);
    }
    const long long ntg = (G + TG - 1) / TG, ntz = (Z + TZ - 1) / TZ;
    const long long ntiles = ntg * ntz;
    const int qg = tid % QG, sg = tid / QG;
    const int q0 = qg * R, m0 = sg * S;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long g0 = (t / ntz) * TG, z0 = (t % ntz) * TZ;
        __syncthreads();
        lt_box<T, LIN, D, TG, TZ, CP, NT, true>(const_cast<T*>(in), sX, G, Z, g0, z0, tid);
        __syncthreads();
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
        lt_box<T, LOUT, M, TG, TZ, CP, NT, false>(out, sX, G, Z, g0, z0, tid);
    }
}

// Generic: run-time M, D and strides; one thread per column q = g*Z + z
// (z fastest), blockDim.x columns per block.  The column's D inputs are
// staged in shared memory with the thread's own loads (coalesced only when z
// is the fastest axis of `in`), L is read from shared memory.
template <class T>
__global__ void __launch_bounds__(128)
ltimes_generic(const T* __restrict__ L, const T* __restrict__ in, T* __restrict__ out, long long G,
               long long Z, int M, int D, long long si_x, long long si_g, long long si_z,
               long long so_x, long long so_g, long long so_z) {
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
        out[m * so_x + g * so_g + z * so_z] = s;
    }
}

}  // namespace cj
#endif
