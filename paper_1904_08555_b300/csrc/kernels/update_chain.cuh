// update_chain.cuh -- batched small-matrix update chain (the Eigen benchmark
// loop of Sec. 5, Listings eigen1/eigen2, in the stable form
// X_{k+1} = X_k + c X_k A_b with X_0 = I and c = 1/(N T)).
//
// Compiled two ways from this one source: by nvcc ahead of time (the generic
// runtime-N kernels and the {4, 8, 16, 32} explicit specializations) and by
// NVRTC at run time for any other (T, N, layout, tile) a caller asks for.
// No includes besides geometry.h, which NVRTC receives from memory.
//
// Row independence: row i of X evolves on its own, x_i <- x_i + c x_i A, so
// one thread can own one row with no communication during the T steps; the
// N threads of an instance read A from shared memory (a broadcast).
#ifndef CJ_UPDATE_CHAIN_CUH
#define CJ_UPDATE_CHAIN_CUH
#include "geometry.h"

namespace cj {

__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// A is invariant across the T steps.  For small N the compiler may keep all
// N*N entries in registers; above that it would hoist them anyway and spill,
// so the base offset is made opaque once per step, which keeps the reads
// inside the step (broadcast shared-memory loads).
template <class T, int N>
struct a_in_regs { static constexpr bool value = sizeof(T) == 8 ? N * N <= 64 : N * N <= 100; };

template <class T>
__device__ __forceinline__ const T* opaque_base(const T* base, int off) {
    asm volatile("" : "+r"(off));
    return base + off;
}

// Stage `ninst` consecutive instances (contiguous in global memory) into
// shared memory as logical row-major matrices with rows of `ar` elements and
// instance pitch P.  Layout 1 stores each instance column-major; it is
// transposed here so that the compute loop is the same for both layouts.
template <class T, int LAYOUT>
__device__ __forceinline__ void chain_stage_in(T* sA, const T* __restrict__ gA, int ninst, int n, int ar,
                                               int P, int tid, int nthreads) {
    const int nn = n * n;
    for (int e = tid; e < ninst * nn; e += nthreads) {
        const int inst = e / nn;
        const int r = e - inst * nn;
        const int row = r / n, col = r - row * n;
        const int l = LAYOUT == 0 ? row : col;
        const int j = LAYOUT == 0 ? col : row;
        sA[inst * P + l * ar + j] = gA[e];
    }
}

// Copy staged results (already in physical order, pitch P) to global memory.
template <class T>
__device__ __forceinline__ void chain_stage_out(T* __restrict__ gX, const T* sA, int ninst, int nn,
                                                int P, int tid, int nthreads) {
    for (int e = tid; e < ninst * nn; e += nthreads) {
        const int inst = e / nn;
        gX[e] = sA[inst * P + (e - inst * nn)];
    }
}

// p += xl * (row of A at `arow`, N entries): 16-byte vector reads when the
// row is padded to a multiple of 4 floats (AR % 4 == 0), scalar otherwise.
template <class T, int N, int AR>
__device__ __forceinline__ void row_axpy(const T* arow, T xl, T (&p)[N]) {
    if constexpr (sizeof(T) == 4 && AR % 4 == 0) {
        const float4* a4 = reinterpret_cast<const float4*>(arow);
#pragma unroll
        for (int q = 0; q < AR / 4; ++q) {
            const float4 v = a4[q];
            const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (4 * q + u < N) p[4 * q + u] = fmaT(xl, w[u], p[4 * q + u]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j) p[j] = fmaT(xl, arow[j], p[j]);
    }
}

// One thread, row i of one instance (A at sA + aoff, logical row-major with
// rows of AR elements): T steps with the row of X in registers.
template <class T, int N, int AR>
__device__ __forceinline__ void row_chain_regs(const T* sA, int aoff, int i, int steps, T cc, T (&x)[N]) {
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = (j == i) ? T(1) : T(0);
    for (int k = 0; k < steps; ++k) {
        const T* a = a_in_regs<T, N>::value ? sA + aoff : opaque_base(sA, aoff);
        T p[N];
#pragma unroll
        for (int j = 0; j < N; ++j) p[j] = T(0);
#pragma unroll
        for (int l = 0; l < N; ++l) row_axpy<T, N, AR>(a + l * AR, x[l], p);
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = fmaT(cc, p[j], x[j]);
    }
}

// Two rows of X per thread (mapping 6, FP32): each 16-byte read of A's row l
// feeds eight fused multiply-adds (four per row).  i1 < 0: the second row is
// absent (odd N) and stays zero.
template <class T, int N, int AR>
__device__ __forceinline__ void row2_chain_regs(const T* sA, int aoff, int i0, int i1, int steps, T cc,
                                                T (&x0)[N], T (&x1)[N]) {
    static_assert(sizeof(T) == 4 && AR % 4 == 0, "mapping 6 is FP32 with rows padded to 16 bytes");
#pragma unroll
    for (int j = 0; j < N; ++j) {
        x0[j] = (j == i0) ? T(1) : T(0);
        x1[j] = (j == i1) ? T(1) : T(0);
    }
    for (int k = 0; k < steps; ++k) {
        const T* a = a_in_regs<T, N>::value ? sA + aoff : opaque_base(sA, aoff);
        T p0[N], p1[N];
#pragma unroll
        for (int j = 0; j < N; ++j) p0[j] = p1[j] = T(0);
#pragma unroll
        for (int l = 0; l < N; ++l) {
            const float4* a4 = reinterpret_cast<const float4*>(a + l * AR);
            const T u0 = x0[l], u1 = x1[l];
#pragma unroll
            for (int q = 0; q < AR / 4; ++q) {
                const float4 v = a4[q];
                const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < N) {
                        p0[4 * q + e] = fmaT(u0, w[e], p0[4 * q + e]);
                        p1[4 * q + e] = fmaT(u1, w[e], p1[4 * q + e]);
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            x0[j] = fmaT(cc, p0[j], x0[j]);
            x1[j] = fmaT(cc, p1[j], x1[j]);
        }
    }
}

// Mapping 6 for N > 32: the two rows of X live in the thread's own
// shared-memory rows xs0 and xs1 (each element read once per N fused
// multiply-adds); the two product rows in registers.
template <class T, int N, int AR>
__device__ __forceinline__ void row2_chain_smem(const T* a, T* xs0, T* xs1, int i0, int i1, int steps, T cc) {
    static_assert(sizeof(T) == 4 && AR % 4 == 0, "mapping 6 is FP32 with rows padded to 16 bytes");
    for (int j = 0; j < N; ++j) {
        xs0[j] = (j == i0) ? T(1) : T(0);
        xs1[j] = (j == i1) ? T(1) : T(0);
    }
    for (int k = 0; k < steps; ++k) {
        T p0[N], p1[N];
#pragma unroll
        for (int j = 0; j < N; ++j) p0[j] = p1[j] = T(0);
#pragma unroll(N > 48 ? 1 : 2)
        for (int l = 0; l < N; ++l) {
            const float4* a4 = reinterpret_cast<const float4*>(a + l * AR);
            const T u0 = xs0[l], u1 = xs1[l];
#pragma unroll
            for (int q = 0; q < AR / 4; ++q) {
                const float4 v = a4[q];
                const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < N) {
                        p0[4 * q + e] = fmaT(u0, w[e], p0[4 * q + e]);
                        p1[4 * q + e] = fmaT(u1, w[e], p1[4 * q + e]);
                    }
            }
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            xs0[j] = fmaT(cc, p0[j], xs0[j]);
            xs1[j] = fmaT(cc, p1[j], xs1[j]);
        }
    }
}

// Same for large N: the row of X lives in the thread's own shared-memory row
// xs (read once per N fused multiply-adds); the product row in registers.
template <class T, int N, int AR>
__device__ __forceinline__ void row_chain_smem(const T* a, T* xs, int i, int steps, T cc) {
    for (int j = 0; j < N; ++j) xs[j] = (j == i) ? T(1) : T(0);
    for (int k = 0; k < steps; ++k) {
        T p[N];
#pragma unroll
        for (int j = 0; j < N; ++j) p[j] = T(0);
#pragma unroll 2
        for (int l = 0; l < N; ++l) row_axpy<T, N, AR>(a + l * AR, xs[l], p);
#pragma unroll
        for (int j = 0; j < N; ++j) xs[j] = fmaT(cc, p[j], xs[j]);
    }
}

// One thread, a whole small instance: X and A in registers.
template <class T, int N>
__device__ __forceinline__ void inst_chain_regs(const T* sa, int steps, T cc, T (&x)[N][N]) {
    T a[N][N];
#pragma unroll
    for (int l = 0; l < N; ++l)
#pragma unroll
        for (int j = 0; j < N; ++j) a[l][j] = sa[l * N + j];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) x[i][j] = (i == j) ? T(1) : T(0);
    for (int k = 0; k < steps; ++k) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T p[N];
#pragma unroll
            for (int j = 0; j < N; ++j) p[j] = T(0);
#pragma unroll
            for (int l = 0; l < N; ++l)
#pragma unroll
                for (int j = 0; j < N; ++j) p[j] = fmaT(x[i][l], a[l][j], p[j]);
#pragma unroll
            for (int j = 0; j < N; ++j) x[i][j] = fmaT(cc, p[j], x[i][j]);
        }
    }
}

// FP64 tensor cores (mapping 4, N a multiple of 8, N <= 32): one warp owns an
// 8-row panel of X and computes P = X_panel A with mma.sync m8n8k4 (FP64 in,
// FP64 accumulate).  Fragment layouts (PTX ISA, m8n8k4 .f64): A operand
// a[r][k] at lane 4r+k; B operand b[k][n] at lane 4n+k; accumulator c[r][n]
// at lane 4r + n/2, component n%2.  X stays in the accumulator layout; the
// A operand of k-block kb (columns 4kb..4kb+3) is gathered from the row's
// owners with two shuffles.  A_b's B fragments are loaded once into
// registers.  The update X += c P is a separate FMA per element, as stated.
__device__ __forceinline__ void dmma_m8n8k4(double (&d)[2], double a, double b) {
    asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

template <int N>
__device__ __forceinline__ void panel_chain_dmma(const double* a_s, int panel, int steps, double cc,
                                                 double (&x)[N / 8][2]) {
    constexpr int NB = N / 8, KB = N / 4;
    const int lane = threadIdx.x & 31, r = lane >> 2, t = lane & 3;
    double b[KB][NB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) b[kb][nb] = a_s[(4 * kb + t) * N + 8 * nb + r];
    const int row = 8 * panel + r;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
        x[nb][0] = (row == 8 * nb + 2 * t) ? 1.0 : 0.0;
        x[nb][1] = (row == 8 * nb + 2 * t + 1) ? 1.0 : 0.0;
    }
    const int base = lane & ~3;
    for (int k = 0; k < steps; ++k) {
        double p[NB][2];
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) p[nb][0] = p[nb][1] = 0.0;
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
            const int src = base | (2 * (kb & 1) + (t >> 1));
            const double v0 = __shfl_sync(0xffffffffu, x[kb >> 1][0], src);
            const double v1 = __shfl_sync(0xffffffffu, x[kb >> 1][1], src);
            const double a = (t & 1) ? v1 : v0;
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) dmma_m8n8k4(p[nb], a, b[kb][nb]);
        }
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
            x[nb][0] = fmaT(cc, p[nb][0], x[nb][0]);
            x[nb][1] = fmaT(cc, p[nb][1], x[nb][1]);
        }
    }
}

// BF16 tensor cores (mapping 3, N >= 16, FP32 state): one warp owns a
// 16-row panel of X (dimensions padded to multiples of 16 with zeros, which
// keeps the padded rows and columns of X at zero) and computes
// P = bf16(X_panel) bf16(A) with mma.sync m16n8k16 (bf16 in, fp32
// accumulate), then X += c P in fp32.  Fragment layouts (PTX ISA, m16n8k16):
// accumulator c0,c1 at (row g, cols 2t, 2t+1), c2,c3 at (row g+8, same
// cols) with g = lane/4, t = lane%4; the A operand of k-tile kt is exactly
// the accumulators of n-tiles 2kt and 2kt+1 rounded to bf16 and packed in
// pairs, so the state never leaves registers.  B operand (A_b): registers
// {A[k=2t][n=g], A[2t+1][g]} and {A[2t+8][g], A[2t+9][g]} per tile.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int N>
__device__ __forceinline__ void panel_chain_bf16(const float* a_s, int panel, int steps, float cc,
                                                 float (&x)[((N + 15) / 16) * 2][4]) {
    constexpr int NP = ((N + 15) / 16) * 16;
    constexpr int KT = NP / 16, NT = NP / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    auto A = [&](int l, int j) -> float { return (l < N && j < N) ? a_s[l * N + j] : 0.f; };
    unsigned b[KT][NT][2];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int n = 8 * j + g, k0 = 16 * kt + 2 * t;
            b[kt][j][0] = pack_bf16(A(k0, n), A(k0 + 1, n));
            b[kt][j][1] = pack_bf16(A(k0 + 8, n), A(k0 + 9, n));
        }
    const int r0 = 16 * panel + g, r1 = r0 + 8;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int c = 8 * j + 2 * t;
        x[j][0] = (r0 < N && r0 == c) ? 1.f : 0.f;
        x[j][1] = (r0 < N && r0 == c + 1) ? 1.f : 0.f;
        x[j][2] = (r1 < N && r1 == c) ? 1.f : 0.f;
        x[j][3] = (r1 < N && r1 == c + 1) ? 1.f : 0.f;
    }
    for (int k = 0; k < steps; ++k) {
        unsigned a[KT][4];
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            a[kt][0] = pack_bf16(x[2 * kt][0], x[2 * kt][1]);
            a[kt][1] = pack_bf16(x[2 * kt][2], x[2 * kt][3]);
            a[kt][2] = pack_bf16(x[2 * kt + 1][0], x[2 * kt + 1][1]);
            a[kt][3] = pack_bf16(x[2 * kt + 1][2], x[2 * kt + 1][3]);
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) mma_bf16_16816(p, a[kt], b[kt][j][0], b[kt][j][1]);
#pragma unroll
            for (int i = 0; i < 4; ++i) x[j][i] = __fmaf_rn(cc, p[i], x[j][i]);
        }
    }
}

// Run the chain for the `ninst` instances staged at sA (pitch per geometry.h)
// and leave each X_T in place of its A, in storage order LAYOUT.
// steps_of(inst) and c_of(inst) give the per-instance T and c.
template <class T, int N, int LAYOUT, int MAP, int IPB, class StepsOf, class COf>
__device__ __forceinline__ void chain_block(T* sA, int ninst, int tid, StepsOf steps_of, COf c_of) {
    constexpr int NN = N * N;
    if constexpr (MAP == 5) {
        // FP32 register blocks: thread (inst, rb, cb) owns rows 4rb..4rb+3 and
        // columns 4cb..4cb+3 of P = X A.  X is kept transposed in shared memory
        // (xt[l][r], pitch NP + 4) so both operands are 16-byte vector reads:
        // 16 FMA per two shared-memory loads.  N is padded to NP, a multiple
        // of 4: A's padded columns are zeroed here, so X's padded rows and
        // columns stay zero.  All threads of the block run the longest
        // instance's step count so every barrier is uniform.
        static_assert(sizeof(T) == 4 && N >= 8, "mapping 5 is FP32 with N >= 8");
        constexpr int NP = (N + 3) / 4 * 4;
        constexpr int P = cjg::chain_pitch(N, 5, 4), AR = cjg::chain_arow(N, 5, 4);
        constexpr int B4 = NP / 4, TPI = B4 * B4, XTP = NP + 4;
        static_assert(AR == NP, "mapping 5 stages A with rows of NP");
        T* xt_all = sA + IPB * P;
        const int inst = tid / TPI, w = tid - inst * TPI;
        const int rb = w % B4, cb = w / B4;
        const bool active = inst < ninst;
        int kmax = 0;
        for (int q = 0; q < ninst; ++q) kmax = max(kmax, steps_of(q));
        const int steps = active ? steps_of(inst) : 0;
        const T cc = active ? c_of(inst) : T(0);
        T* xt = xt_all + (active ? inst : 0) * NP * XTP;
        T* a_w = sA + (active ? inst : 0) * P;
        const T* a = a_w;
        if (active) {
            for (int e = w; e < NP * NP; e += TPI) {
                const int l = e / NP, r = e - l * NP;
                xt[l * XTP + r] = (l == r && l < N) ? T(1) : T(0);
            }
            if constexpr (NP != N)
                for (int e = w; e < N * (NP - N); e += TPI) {
                    const int l = e / (NP - N), j = N + (e - l * (NP - N));
                    a_w[l * NP + j] = T(0);
                }
        }
        __syncthreads();
        for (int k = 0; k < kmax; ++k) {
            float acc[4][4] = {};
            const bool run = k < steps;
            if (run) {
#pragma unroll 4
                for (int l = 0; l < N; ++l) {
                    const float4 xv = *reinterpret_cast<const float4*>(xt + l * XTP + 4 * rb);
                    const float4 av = *reinterpret_cast<const float4*>(a + l * NP + 4 * cb);
                    const float xr[4] = {xv.x, xv.y, xv.z, xv.w};
                    const float ar[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaT(xr[i], ar[j], acc[i][j]);
                }
            }
            __syncthreads();   // every read of X_k is done
            if (run) {
                // column 4cb + j of X^T, rows 4rb..4rb+3: one 16-byte read and
                // write each (a warp's four-row runs are contiguous)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float4* xp = reinterpret_cast<float4*>(xt + (4 * cb + j) * XTP + 4 * rb);
                    float4 v = *xp;
                    v.x = fmaT(cc, acc[0][j], v.x);
                    v.y = fmaT(cc, acc[1][j], v.y);
                    v.z = fmaT(cc, acc[2][j], v.z);
                    v.w = fmaT(cc, acc[3][j], v.w);
                    *xp = v;
                }
            }
            __syncthreads();   // X_{k+1} complete
        }
        // X_T into the staging area in storage order (A is no longer needed)
        if (active)
            for (int e = w; e < NN; e += TPI) {
                const int i = e / N, j = e - i * N;
                sA[inst * P + (LAYOUT == 0 ? i * N + j : j * N + i)] = xt[j * XTP + i];
            }
    } else if constexpr (MAP == 8) {
        // FP32 register blocks of 4 rows x 8 columns of P = X A: thread
        // (inst, rb, cb) owns rows 4rb..4rb+3 and columns 8cb..8cb+7, so each
        // k step of the product is one 16-byte read of X^T and two of A for
        // 32 fused multiply-adds (mapping 5: two reads for 16).  Rows are
        // padded to NR (a multiple of 4), columns to NC (a multiple of 8); X^T
        // is kept in shared memory as xt[l][r] with NC rows of pitch NR + 4,
        // twice: step k reads X_k from one copy and writes X_{k+1} into the
        // other, so a step needs one barrier (mapping 5: two).  A's padded
        // columns are zeroed here, so P's padded columns, and with them X's
        // padded rows and columns, stay exactly zero; the product runs over
        // the N real k only.  Each copy is chain_m8_xti(N) elements (an odd
        // number of 16-byte units).  All threads of the block run the longest
        // instance's step count so every barrier is uniform; an instance's
        // X_T is in copy T % 2.
        static_assert(sizeof(T) == 4 && N >= 8, "mapping 8 is FP32 with N >= 8");
        constexpr int NR = (N + 3) / 4 * 4, NC = (N + 7) / 8 * 8;
        constexpr int P = cjg::chain_pitch(N, 8, 4), AR = cjg::chain_arow(N, 8, 4);
        constexpr int B4 = NR / 4, B8 = NC / 8, TPI = B4 * B8, XTP = NR + 4, XTI = cjg::chain_m8_xti(N);
        static_assert(AR == NC, "mapping 8 stages A with rows of NC");
        T* xt_all = sA + IPB * P;
        const int inst = tid / TPI, w = tid - inst * TPI;
        const int rb = w % B4, cb = w / B4;
        const bool active = inst < ninst;
        int kmax = 0;
        for (int q = 0; q < ninst; ++q) kmax = max(kmax, steps_of(q));
        const int steps = active ? steps_of(inst) : 0;
        const T cc = active ? c_of(inst) : T(0);
        T* xt0 = xt_all + (active ? inst : 0) * 2 * XTI;   // X_k for even k
        T* xt1 = xt0 + XTI;                                // odd k
        T* a_w = sA + (active ? inst : 0) * P;
        const T* a = a_w;
        if (active) {
            // X_0 = I; every entry of the other copy is written by the first step
            for (int e = w; e < NC * NR; e += TPI) {
                const int l = e / NR, r = e - l * NR;
                xt0[l * XTP + r] = (l == r && l < N) ? T(1) : T(0);
            }
            if constexpr (NC != N)
                for (int e = w; e < N * (NC - N); e += TPI) {
                    const int l = e / (NC - N), j = N + (e - l * (NC - N));
                    a_w[l * NC + j] = T(0);
                }
        }
        __syncthreads();
        for (int k = 0; k < kmax; ++k) {
            const T* cur = (k & 1) ? xt1 : xt0;
            T* nxt = (k & 1) ? xt0 : xt1;
            if (k < steps) {
                float acc[4][8] = {};
#pragma unroll 4
                for (int l = 0; l < N; ++l) {
                    const float4 xv = *reinterpret_cast<const float4*>(cur + l * XTP + 4 * rb);
                    const float4 a0 = *reinterpret_cast<const float4*>(a + l * NC + 8 * cb);
                    const float4 a1 = *reinterpret_cast<const float4*>(a + l * NC + 8 * cb + 4);
                    const float xr[4] = {xv.x, xv.y, xv.z, xv.w};
                    const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaT(xr[i], ar[j], acc[i][j]);
                }
                // column 8cb + j of X_{k+1}^T, rows 4rb..4rb+3: one 16-byte read of X_k and one write
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float4 v = *reinterpret_cast<const float4*>(cur + (8 * cb + j) * XTP + 4 * rb);
                    v.x = fmaT(cc, acc[0][j], v.x);
                    v.y = fmaT(cc, acc[1][j], v.y);
                    v.z = fmaT(cc, acc[2][j], v.z);
                    v.w = fmaT(cc, acc[3][j], v.w);
                    *reinterpret_cast<float4*>(nxt + (8 * cb + j) * XTP + 4 * rb) = v;
                }
            }
            __syncthreads();   // X_{k+1} complete, and every read of X_k done before it is overwritten
        }
        // X_T into the staging area in storage order (A is no longer needed)
        const T* xf = (steps & 1) ? xt1 : xt0;
        if (active)
            for (int e = w; e < NN; e += TPI) {
                const int i = e / N, j = e - i * N;
                sA[inst * P + (LAYOUT == 0 ? i * N + j : j * N + i)] = xf[j * XTP + i];
            }
    } else if constexpr (MAP == 6) {
        static_assert(sizeof(T) == 4, "mapping 6 is FP32");
        constexpr int P = cjg::chain_pitch(N, 6, 4), AR = cjg::chain_arow(N, 6, 4), H = (N + 1) / 2;
        const int inst = tid / H, h = tid - inst * H;
        const bool active = inst < ninst;
        const int i1 = h + H < N ? h + H : -1;
        if constexpr (N <= 32) {
            T x0[N], x1[N];
            if (active) row2_chain_regs<T, N, AR>(sA, inst * P, h, i1, steps_of(inst), c_of(inst), x0, x1);
            __syncthreads();
            if (active) {
#pragma unroll
                for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? h * N + j : j * N + h)] = x0[j];
                if (i1 >= 0) {
#pragma unroll
                    for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? i1 * N + j : j * N + i1)] = x1[j];
                }
            }
        } else {
            constexpr int XP = cjg::xrow_pitch(N);
            T* xs0 = sA + IPB * P + (2 * tid) * XP;
            T* xs1 = xs0 + XP;
            if (active) row2_chain_smem<T, N, AR>(sA + inst * P, xs0, xs1, h, i1, steps_of(inst), c_of(inst));
            __syncthreads();
            if (active) {
                for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? h * N + j : j * N + h)] = xs0[j];
                if (i1 >= 0)
                    for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? i1 * N + j : j * N + i1)] = xs1[j];
            }
        }
    } else if constexpr (MAP == 3) {
        static_assert(sizeof(T) == 4 && N >= 16, "mapping 3 is bf16 operands with fp32 state, N >= 16");
        constexpr int P = cjg::row_pitch(NN, 4);
        constexpr int NPAN = (N + 15) / 16;
        const int warp = tid >> 5;
        const int inst = warp / NPAN, panel = warp - inst * NPAN;
        const bool active = inst < ninst;   // uniform across the warp
        float x[NPAN * 2][4];
        if (active) panel_chain_bf16<N>(sA + inst * P, panel, steps_of(inst), (float)c_of(inst), x);
        __syncthreads();
        if (active) {
            const int lane = tid & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
            for (int j = 0; j < NPAN * 2; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int row = 16 * panel + g + (i >= 2 ? 8 : 0), col = 8 * j + 2 * t + (i & 1);
                    if (row < N && col < N) sA[inst * P + (LAYOUT == 0 ? row * N + col : col * N + row)] = x[j][i];
                }
        }
    } else if constexpr (MAP == 4) {
        static_assert(sizeof(T) == 8 && N % 8 == 0 && N <= 32, "mapping 4 is FP64 with N = 8, 16, 24, 32");
        constexpr int P = cjg::row_pitch(NN, 8);
        constexpr int NB = N / 8;
        const int warp = tid >> 5;
        const int inst = warp / NB, panel = warp - inst * NB;
        const bool active = inst < ninst;   // uniform across the warp
        double x[NB][2];
        if (active) panel_chain_dmma<N>(sA + inst * P, panel, steps_of(inst), c_of(inst), x);
        __syncthreads();
        if (active) {
            const int lane = tid & 31, row = 8 * panel + (lane >> 2), t = lane & 3;
#pragma unroll
            for (int nb = 0; nb < NB; ++nb)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int col = 8 * nb + 2 * t + i;
                    sA[inst * P + (LAYOUT == 0 ? row * N + col : col * N + row)] = x[nb][i];
                }
        }
    } else if constexpr (MAP == 2) {
        constexpr int P = cjg::inst_pitch(NN);
        const bool active = tid < ninst;
        T x[N][N];
        if (active) inst_chain_regs<T, N>(sA + tid * P, steps_of(tid), c_of(tid), x);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int j = 0; j < N; ++j) sA[tid * P + (LAYOUT == 0 ? i * N + j : j * N + i)] = x[i][j];
        }
    } else {
        constexpr int P = cjg::chain_pitch(N, 1, (int)sizeof(T));
        constexpr int AR = cjg::chain_arow(N, 1, (int)sizeof(T));
        constexpr bool XREG = N <= cjg::chain_reg_rows_max((int)sizeof(T));
        const int inst = tid / N;
        const int i = tid - inst * N;
        const bool active = inst < ninst;
        if constexpr (XREG) {
            T x[N];
            if (active) row_chain_regs<T, N, AR>(sA, inst * P, i, steps_of(inst), c_of(inst), x);
            __syncthreads();
            if (active) {
#pragma unroll
                for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? i * N + j : j * N + i)] = x[j];
            }
        } else {
            constexpr int XP = cjg::xrow_pitch(N);
            T* xs = sA + IPB * P + tid * XP;
            if (active) row_chain_smem<T, N, AR>(sA + inst * P, xs, i, steps_of(inst), c_of(inst));
            __syncthreads();
            if (active)
                for (int j = 0; j < N; ++j) sA[inst * P + (LAYOUT == 0 ? i * N + j : j * N + i)] = xs[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Specialized kernel.  MAP 1: one thread per row of X, A in shared memory.
// MAP 2: one thread per instance, X and A in registers (small N).
// A block is shaped for IPB instances; it takes ipb (1 <= ipb <= IPB) of
// them, so that a batch too small to fill the SMs with whole blocks can be
// spread over more blocks (the host picks ipb per launch).
// ---------------------------------------------------------------------------
template <class T, int N, int LAYOUT, int MAP, int IPB>
__global__ void __launch_bounds__(cjg::chain_threads(N, MAP, IPB))
update_chain(const T* __restrict__ A, T* __restrict__ X, long long batch, int steps, double c, int ipb) {
    constexpr int NN = N * N;
    constexpr int NT = cjg::chain_threads(N, MAP, IPB);
    constexpr int P = cjg::chain_pitch(N, MAP, (int)sizeof(T));
    constexpr int AR = cjg::chain_arow(N, MAP, (int)sizeof(T));
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sA = reinterpret_cast<T*>(cj_smem);
    ipb = ipb < 1 ? 1 : ipb > IPB ? IPB : ipb;
    const long long b0 = (long long)blockIdx.x * ipb;
    if (b0 >= batch) return;
    const int ninst = (batch - b0) < ipb ? (int)(batch - b0) : ipb;
    const T cc = (T)c;
    const int tid = threadIdx.x;
    chain_stage_in<T, LAYOUT>(sA, A + b0 * NN, ninst, N, AR, P, tid, NT);
    __syncthreads();
    chain_block<T, N, LAYOUT, MAP, IPB>(
        sA, ninst, tid, [&](int) { return steps; }, [&](int) { return cc; });
    __syncthreads();
    chain_stage_out<T>(X + b0 * NN, sA, ninst, NN, P, tid, NT);
}

// ---------------------------------------------------------------------------
// Generic runtime-N kernel (the analog of Eigen's Dynamic-size matrices): the
// same one-thread-per-row mapping, but N, the layout and the instances per
// block are run-time values, so the thread's row of X and of the product live
// in shared memory and every loop has run-time bounds.  Supports 1 <= n <= 64.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void generic_row_chain(const T* a, T* xs, T* ps, int n, int i, int steps, T cc) {
    for (int j = 0; j < n; ++j) xs[j] = (j == i) ? T(1) : T(0);
    for (int k = 0; k < steps; ++k) {
        for (int j = 0; j < n; ++j) {
            T s = T(0);
            for (int l = 0; l < n; ++l) s = fmaT(xs[l], a[l * n + j], s);
            ps[j] = s;
        }
        for (int j = 0; j < n; ++j) xs[j] = fmaT(cc, ps[j], xs[j]);
    }
}

template <class T>
__global__ void __launch_bounds__(256)
update_chain_generic(const T* __restrict__ A, T* __restrict__ X, long long batch, int steps,
                     double c, int n, int layout, int ipb) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sA = reinterpret_cast<T*>(cj_smem);
    const int nn = n * n;
    const int P = cjg::row_pitch(nn, (int)sizeof(T));
    const int XP = cjg::xrow_pitch(n);
    const int nthreads = blockDim.x;
    const int tid = threadIdx.x;
    T* xs = sA + ipb * P + tid * XP;
    T* ps = sA + ipb * P + nthreads * XP + tid * XP;
    const long long b0 = (long long)blockIdx.x * ipb;
    if (b0 >= batch) return;
    const int ninst = (batch - b0) < ipb ? (int)(batch - b0) : ipb;
    if (layout == 0) chain_stage_in<T, 0>(sA, A + b0 * nn, ninst, n, n, P, tid, nthreads);
    else             chain_stage_in<T, 1>(sA, A + b0 * nn, ninst, n, n, P, tid, nthreads);
    __syncthreads();
    const int inst = tid / n;
    const int i = tid - inst * n;
    const bool active = inst < ninst;
    if (active) generic_row_chain<T>(sA + inst * P, xs, ps, n, i, steps, (T)c);
    __syncthreads();
    if (active)
        for (int j = 0; j < n; ++j) sA[inst * P + (layout == 0 ? i * n + j : j * n + i)] = xs[j];
    __syncthreads();
    chain_stage_out<T>(X + b0 * nn, sA, ninst, nn, P, tid, nthreads);
}

// ---------------------------------------------------------------------------
// The paper's literal Eigen benchmark recurrence (Sec. 5, Listing eigen1):
//     M_{k+1} = Ones + c (M_k + M_k M_k),   k = 0 .. R-1,   per instance,
// the listing's case being c = 5e-5 and M_0(i, j) = i + N j, which the caller
// passes.  Unlike the update chain, row i of M_{k+1} needs every row of M_k,
// so a block keeps M_k of each of its instances in shared memory (two
// buffers, padded rows and instances, one barrier per step); thread (instance, i) keeps
// its own row in registers and reads the other rows as broadcasts.  Each
// element is formed as 1 + c * (m + q) with a separate multiply and add, the
// order the listing writes.  Row-major.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double eig_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float eig_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double eig_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float eig_add(float a, float b) { return __fadd_rn(a, b); }

// Instances [0, ninst) of a block between global memory (contiguous, row-major)
// and a shared-memory buffer with rows of eig_rp(n, sizeof(T)) and instances
// ip elements apart.
template <class T>
__device__ __forceinline__ void eig_load(T* buf, const T* __restrict__ g, int ninst, int n, int ip, int tid,
                                         int nthreads) {
    const int rp = cjg::eig_rp(n, (int)sizeof(T)), nn = n * n;
    for (int e = tid; e < ninst * nn; e += nthreads) {
        const int inst = e / nn, r = e - inst * nn, i = r / n;
        buf[inst * ip + i * rp + (r - i * n)] = g[e];
    }
}
template <class T>
__device__ __forceinline__ void eig_store(T* __restrict__ g, const T* buf, int ninst, int n, int ip, int tid,
                                          int nthreads) {
    const int rp = cjg::eig_rp(n, (int)sizeof(T)), nn = n * n;
    for (int e = tid; e < ninst * nn; e += nthreads) {
        const int inst = e / nn, r = e - inst * nn, i = r / n;
        g[e] = buf[inst * ip + i * rp + (r - i * n)];
    }
}

template <class T, int N, int IPB>
__global__ void __launch_bounds__(cjg::chain_threads(N, 1, IPB))
eigen_recurrence(const T* __restrict__ M0, T* __restrict__ M, long long batch, int repeat, double c) {
    constexpr int NN = N * N, NT = cjg::chain_threads(N, 1, IPB), RP = cjg::eig_rp(N, (int)sizeof(T)),
                  P = cjg::eig_ip(N, (int)sizeof(T));
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* cur = reinterpret_cast<T*>(cj_smem);
    T* nxt = cur + IPB * P;
    const long long b0 = (long long)blockIdx.x * IPB;
    if (b0 >= batch) return;
    const int ninst = (batch - b0) < IPB ? (int)(batch - b0) : IPB;
    const int tid = threadIdx.x;
    eig_load<T>(cur, M0 + b0 * NN, ninst, N, P, tid, NT);
    __syncthreads();
    const int inst = tid / N, i = tid - inst * N;
    const bool active = inst < ninst;
    const T cc = (T)c;
    T x[N];
    if (active) {
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = cur[inst * P + i * RP + j];
    }
    for (int k = 0; k < repeat; ++k) {
        if (active) {
            const T* m = opaque_base(cur, inst * P);
            T q[N];
#pragma unroll
            for (int j = 0; j < N; ++j) q[j] = T(0);
#pragma unroll
            for (int l = 0; l < N; ++l) {
                const T xl = x[l];
                // row l of M_k (a broadcast within the instance) in 16-byte vectors
                constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
                for (int q4 = 0; q4 < (N + V - 1) / V; ++q4) {
                    T w[V];
                    if constexpr (V == 4) {
                        const float4 t = reinterpret_cast<const float4*>(m + l * RP)[q4];
                        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
                    } else {
                        const double2 t = reinterpret_cast<const double2*>(m + l * RP)[q4];
                        w[0] = t.x; w[1] = t.y;
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (V * q4 + e < N) q[V * q4 + e] = fmaT(xl, w[e], q[V * q4 + e]);
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                x[j] = eig_add(T(1), eig_mul(cc, eig_add(x[j], q[j])));
                nxt[inst * P + i * RP + j] = x[j];
            }
        }
        __syncthreads();   // M_{k+1} complete; M_k no longer read
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    eig_store<T>(M + b0 * NN, cur, ninst, N, P, tid, NT);
}

// Two rows per thread (tile mapping 2, FP32): thread (instance, h) forms rows
// h and h + ceil(N / 2) of M_{k+1}, so every element of row l read from
// shared memory feeds two multiply-adds instead of one; the one-row kernel is
// bound by shared-memory wavefronts at N >= 9.  Per element the operations
// and their order are the one-row kernel's (l ascending, one FMA per term,
// then 1 + c (m + q) with a separate multiply and add), so the results are the
// same bit for bit.  The thread of a half-row (h = ceil(N / 2) - 1, N odd)
// has no second row; it runs the same loop with zeros and stores one row.
template <class T, int N, int IPB>
__global__ void __launch_bounds__(cjg::chain_threads(N, 6, IPB))
eigen_recurrence2(const T* __restrict__ M0, T* __restrict__ M, long long batch, int repeat, double c) {
    constexpr int H = (N + 1) / 2, NN = N * N, NT = cjg::chain_threads(N, 6, IPB),
                  RP = cjg::eig_rp(N, (int)sizeof(T)), P = cjg::eig_ip(N, (int)sizeof(T), 2);
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* cur = reinterpret_cast<T*>(cj_smem);
    T* nxt = cur + IPB * P;
    const long long b0 = (long long)blockIdx.x * IPB;
    if (b0 >= batch) return;
    const int ninst = (batch - b0) < IPB ? (int)(batch - b0) : IPB;
    const int tid = threadIdx.x;
    eig_load<T>(cur, M0 + b0 * NN, ninst, N, P, tid, NT);
    __syncthreads();
    const int inst = tid / H, h = tid - inst * H;
    const bool active = inst < ninst;
    const bool two = h + H < N;
    const T cc = (T)c;
    T x0[N], x1[N];
    if (active) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            x0[j] = cur[inst * P + h * RP + j];
            x1[j] = two ? cur[inst * P + (h + H) * RP + j] : T(0);
        }
    }
    for (int k = 0; k < repeat; ++k) {
        if (active) {
            const T* m = opaque_base(cur, inst * P);
            T q0[N], q1[N];
#pragma unroll
            for (int j = 0; j < N; ++j) q0[j] = q1[j] = T(0);
#pragma unroll
            for (int l = 0; l < N; ++l) {
                const T xl0 = x0[l], xl1 = x1[l];
                constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
                for (int q4 = 0; q4 < (N + V - 1) / V; ++q4) {
                    T w[V];
                    if constexpr (V == 4) {
                        const float4 t = reinterpret_cast<const float4*>(m + l * RP)[q4];
                        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
                    } else {
                        const double2 t = reinterpret_cast<const double2*>(m + l * RP)[q4];
                        w[0] = t.x; w[1] = t.y;
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (V * q4 + e < N) {
                            q0[V * q4 + e] = fmaT(xl0, w[e], q0[V * q4 + e]);
                            q1[V * q4 + e] = fmaT(xl1, w[e], q1[V * q4 + e]);
                        }
                }
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                x0[j] = eig_add(T(1), eig_mul(cc, eig_add(x0[j], q0[j])));
                nxt[inst * P + h * RP + j] = x0[j];
            }
            if (two) {
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    x1[j] = eig_add(T(1), eig_mul(cc, eig_add(x1[j], q1[j])));
                    nxt[inst * P + (h + H) * RP + j] = x1[j];
                }
            }
        }
        __syncthreads();   // M_{k+1} complete; M_k no longer read
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    eig_store<T>(M + b0 * NN, cur, ninst, N, P, tid, NT);
}

// Generic: run-time n (1..64) and instances per block; every row in shared memory.
template <class T>
__global__ void __launch_bounds__(256)
eigen_recurrence_generic(const T* __restrict__ M0, T* __restrict__ M, long long batch, int repeat, double c, int n,
                         int ipb) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    const int rp = cjg::eig_rp(n, (int)sizeof(T)), p = cjg::eig_ip(n, (int)sizeof(T)), nn = n * n;
    T* cur = reinterpret_cast<T*>(cj_smem);
    T* nxt = cur + ipb * p;
    const long long b0 = (long long)blockIdx.x * ipb;
    if (b0 >= batch) return;
    const int ninst = (batch - b0) < ipb ? (int)(batch - b0) : ipb;
    const int tid = threadIdx.x, nthreads = blockDim.x;
    eig_load<T>(cur, M0 + b0 * nn, ninst, n, p, tid, nthreads);
    __syncthreads();
    const int inst = tid / n, i = tid - inst * n;
    const bool active = inst < ninst;
    const T cc = (T)c;
    for (int k = 0; k < repeat; ++k) {
        if (active) {
            const T* m = cur + inst * p;
            for (int j = 0; j < n; ++j) {
                T s = T(0);
                for (int l = 0; l < n; ++l) s = fmaT(m[i * rp + l], m[l * rp + j], s);
                nxt[inst * p + i * rp + j] = eig_add(T(1), eig_mul(cc, eig_add(m[i * rp + j], s)));
            }
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
    }
    eig_store<T>(M + b0 * nn, cur, ninst, n, p, tid, nthreads);
}

// ---------------------------------------------------------------------------
// One chunk of a grouped work list: `ninst` (<= IPB) consecutive items, each
// {element offset of A and X in the pools, T, reserved} as int64, staged in,
// run, staged out by a block of `nt` threads (nt >= the mapping's thread
// count; threads past it take every barrier but no work).  c = 1/(N T) is
// formed per instance in double, as the host would.  Row-major only.
// Returns after a final barrier, so the caller may reuse shared memory.
// ---------------------------------------------------------------------------
template <class T, int N, int MAP, int IPB>
__device__ __forceinline__ void grouped_chunk(const long long* __restrict__ items, int ninst,
                                              const T* __restrict__ A_pool, T* __restrict__ X_pool, T* sA,
                                              long long* s_off, int* s_steps, int tid, int nt) {
    constexpr int NN = N * N;
    constexpr int P = cjg::chain_pitch(N, MAP, (int)sizeof(T));
    constexpr int AR = cjg::chain_arow(N, MAP, (int)sizeof(T));
    for (int q = tid; q < ninst; q += nt) {
        s_off[q] = items[3 * q];
        s_steps[q] = (int)items[3 * q + 1];
    }
    __syncthreads();
    for (int e = tid; e < ninst * NN; e += nt) {
        const int inst = e / NN, r = e - inst * NN;
        const int row = r / N, col = r - row * N;
        sA[inst * P + row * AR + col] = A_pool[s_off[inst] + r];
    }
    __syncthreads();
    chain_block<T, N, 0, MAP, IPB>(
        sA, ninst, tid, [&](int q) { return s_steps[q]; },
        [&](int q) { return (T)(1.0 / ((double)N * (double)s_steps[q])); });
    __syncthreads();
    for (int e = tid; e < ninst * NN; e += nt) {
        const int inst = e / NN;
        X_pool[s_off[inst] + (e - inst * NN)] = sA[inst * P + (e - inst * NN)];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Grouped persistent kernel: instances of one size N with different step
// counts, listed in a work list (sorted by T descending by the host).  Each
// block repeatedly takes the next chunk of IPB consecutive items from a
// device counter (atomicAdd) until the list is exhausted.
// ---------------------------------------------------------------------------
template <class T, int N, int MAP, int IPB>
__global__ void __launch_bounds__(cjg::chain_threads(N, MAP, IPB))
update_chain_grouped(const long long* __restrict__ items, const T* __restrict__ A_pool,
                     T* __restrict__ X_pool, int* __restrict__ counter, long long n_items) {
    constexpr int NT = cjg::chain_threads(N, MAP, IPB);
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sA = reinterpret_cast<T*>(cj_smem);
    __shared__ long long s_off[IPB];
    __shared__ int s_steps[IPB];
    __shared__ int s_chunk;
    const int tid = threadIdx.x;
    const long long n_chunks = (n_items + IPB - 1) / IPB;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(counter, 1);
        __syncthreads();
        const long long chunk = s_chunk;
        if (chunk >= n_chunks) break;
        const long long it0 = chunk * IPB;
        const int ninst = (n_items - it0) < IPB ? (int)(n_items - it0) : IPB;
        grouped_chunk<T, N, MAP, IPB>(items + 3 * it0, ninst, A_pool, X_pool, sA, s_off, s_steps, tid, NT);
    }
}

// A group's chunk body as a separate function, for the plan dispatcher: each
// body keeps its own register allocation (inlined into one switch, the bodies'
// live ranges would be allocated together and spill).
template <class T, int N, int MAP, int IPB, int NT>
__device__ __noinline__ void grouped_chunk_call(const long long* __restrict__ items, int ninst,
                                                const T* __restrict__ A_pool, T* __restrict__ X_pool, T* sA,
                                                long long* s_off, int* s_steps) {
    grouped_chunk<T, N, MAP, IPB>(items, ninst, A_pool, X_pool, sA, s_off, s_steps, threadIdx.x, NT);
}

// ---------------------------------------------------------------------------
// Plan dispatcher: one persistent launch for a whole uneven batch.  The host
// generates, per plan, a kernel whose body is a switch over the plan's groups
// (one grouped_chunk instantiation per group, all for the same block size)
// and a ticket list: each ticket is one chunk of one group, {first item,
// (group << 16) | item count}, ordered by cost T N^3 descending, so the
// longest chunks start first and the short ones fill the tail.  Blocks take
// tickets from one counter until the list is exhausted.  `body(group, items,
// ninst, sA, s_off, s_steps)` runs one chunk; it must take the same barriers
// on every thread of the block.
// ---------------------------------------------------------------------------
template <class T, class Body>
__device__ __forceinline__ void dispatch_tickets(const long long* __restrict__ tickets, int n_tickets,
                                                 const long long* __restrict__ items, int* __restrict__ counter,
                                                 Body body) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    T* sA = reinterpret_cast<T*>(cj_smem);
    __shared__ long long s_off[256];
    __shared__ int s_steps[256];
    __shared__ int s_ticket;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_ticket;
        if (t >= n_tickets) break;
        const long long first = tickets[2 * t];
        const int gc = (int)tickets[2 * t + 1];
        body(gc >> 16, items + 3 * first, gc & 0xffff, sA, s_off, s_steps);
    }
}

// Generic grouped kernel: the stand-in for update_chain_grouped while its
// specialization compiles.  Run-time n and instances per chunk (ipb <= 256);
// rows of X and of the product in shared memory.
template <class T>
__global__ void __launch_bounds__(256)
update_chain_grouped_generic(const long long* __restrict__ items, const T* __restrict__ A_pool,
                             T* __restrict__ X_pool, int* __restrict__ counter, long long n_items,
                             int n, int ipb) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    __shared__ long long s_off[256];
    __shared__ int s_steps[256];
    __shared__ int s_chunk;
    T* sA = reinterpret_cast<T*>(cj_smem);
    const int nn = n * n;
    const int P = cjg::row_pitch(nn, (int)sizeof(T));
    const int XP = cjg::xrow_pitch(n);
    const int nthreads = blockDim.x;
    const int tid = threadIdx.x;
    T* xs = sA + ipb * P + tid * XP;
    T* ps = sA + ipb * P + nthreads * XP + tid * XP;
    const long long n_chunks = (n_items + ipb - 1) / ipb;
    for (;;) {
        if (tid == 0) s_chunk = atomicAdd(counter, 1);
        __syncthreads();
        const long long chunk = s_chunk;
        if (chunk >= n_chunks) break;
        const long long it0 = chunk * ipb;
        const int ninst = (n_items - it0) < ipb ? (int)(n_items - it0) : ipb;
        for (int q = tid; q < ninst; q += nthreads) {
            s_off[q] = items[3 * (it0 + q)];
            s_steps[q] = (int)items[3 * (it0 + q) + 1];
        }
        __syncthreads();
        for (int e = tid; e < ninst * nn; e += nthreads) {
            const int inst = e / nn;
            sA[inst * P + (e - inst * nn)] = A_pool[s_off[inst] + (e - inst * nn)];
        }
        __syncthreads();
        const int inst = tid / n;
        const int i = tid - inst * n;
        const bool active = inst < ninst;
        if (active) {
            const int steps = s_steps[inst];
            generic_row_chain<T>(sA + inst * P, xs, ps, n, i, steps, (T)(1.0 / ((double)n * (double)steps)));
        }
        __syncthreads();
        if (active)
            for (int j = 0; j < n; ++j) sA[inst * P + i * n + j] = xs[j];
        __syncthreads();
        for (int e = tid; e < ninst * nn; e += nthreads) {
            const int inst2 = e / nn;
            X_pool[s_off[inst2] + (e - inst2 * nn)] = sA[inst2 * P + (e - inst2 * nn)];
        }
        __syncthreads();
    }
}

}  // namespace cj
#endif
