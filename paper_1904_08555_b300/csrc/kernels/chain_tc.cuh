// chain_tc.cuh -- the BF16 update chain on the 5th-generation tensor cores
// (tile mapping 7): per instance X_0 = I, X_{k+1} = X_k + c X_k A with the
// product P = bf16(X_k) bf16(A) formed by tcgen05.mma (kind::f16, FP32
// accumulator in tensor memory) and the state X kept in FP32 registers.
//
// One instance at a time per CTA of 128 threads.  Thread r owns row r of X
// (rows r >= N are zero padding: the MMA's M is 128).  Per step:
//   1. every thread with r < N writes bf16(row r) into the A operand (shared
//      memory, K-major core matrices);
//   2. one thread issues NP / 16 MMAs (K = 16 each) into the accumulator and
//      commits them to an mbarrier;
//   3. all threads wait on it (bounded), read their accumulator row with
//      tcgen05.ld (warp w reads lanes 32w..32w+31) and update X += c P.
// The B operand, A^T in bf16, is staged once per instance.  NP = N rounded
// up to 16; padded rows and columns are zero, so X's padding stays zero.
//
// Operand layout (both operands, K-major, no swizzle): 8-row x 16-byte core
// matrices (8 bf16 along K), K-adjacent ones 128 B apart (LBO), 8-row groups
// NP / 8 * 128 B apart (SBO).  Instruction descriptor: FP32 D, BF16 A and B,
// both K-major, N = NP (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24).
//
// Every wait is bounded (about a second, as in the LTimes tensor-core
// kernel): on expiry the block stops computing, stays in step with its
// barriers, counts the event once in cj_wait_timeouts, frees its tensor
// memory and returns; its remaining outputs are not written.
#ifndef CJ_CHAIN_TC_CUH
#define CJ_CHAIN_TC_CUH
#include "ltimes.cuh"
#include "update_chain.cuh"

namespace cj {

// Byte offset of (row, k) in a K-major bf16 operand of K extent NP.
template <int NP>
__device__ __forceinline__ unsigned ctc_off(int row, int k) {
    return (unsigned)((row >> 3) * (NP / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void ctc_mma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                             unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Per-CTA state of the tensor-core chain: shared-memory operands, the tensor
// memory columns, the MMA-completion mbarrier and its phase, the abort flag.
template <int N>
struct ChainTC {
    static constexpr int NP = (N + 15) / 16 * 16;
    static constexpr int TCOLS = NP <= 32 ? 32 : NP <= 64 ? 64 : 128;
    static constexpr unsigned A_BYTES = 128u * NP * 2u, SBO = NP / 8 * 128u;
    static constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NP >> 3) << 17) |
                                      ((128u >> 4) << 24);
    unsigned a_u, b_u, tmem, bar;
    int phase;
    bool aborted;
};

// Set up a CTA (all 128 threads): zero the A operand (its padding rows stay
// zero), allocate tensor memory, initialise the mbarrier.
template <int N>
__device__ __forceinline__ void chain_tc_setup(ChainTC<N>& s, unsigned char* smem, unsigned long long* bar,
                                               unsigned* tmem_slot) {
    const int tid = threadIdx.x;
    s.a_u = lt_smem_u32(smem);
    s.b_u = s.a_u + ChainTC<N>::A_BYTES;
    for (unsigned e = tid; e < ChainTC<N>::A_BYTES / 16; e += 128) reinterpret_cast<uint4*>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        lt_mbar_init(lt_smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(lt_smem_u32(tmem_slot)),
                     "r"(ChainTC<N>::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    lt_tc_fence_before();
    __syncthreads();
    lt_tc_fence_after();
    s.tmem = *tmem_slot;
    s.bar = lt_smem_u32(bar);
    s.phase = 0;
    s.aborted = false;
}

// One instance: A (logical row-major when LAYOUT == 0, column-major when 1)
// in, X_T out in the same layout.  Every thread of the CTA calls it.
template <int N, int LAYOUT>
__device__ __forceinline__ void chain_tc_instance(ChainTC<N>& s, unsigned char* smem, const float* __restrict__ A,
                                                  float* __restrict__ X, int steps, float cc) {
    constexpr int NP = ChainTC<N>::NP;
    const int tid = threadIdx.x, warp = tid >> 5;
    // B operand: B[n][k] = A[k][n] (the product is X A), zero-padded to NP x NP
    unsigned short* bs = reinterpret_cast<unsigned short*>(smem + ChainTC<N>::A_BYTES);
    for (int e = tid; e < NP * NP; e += 128) {
        const int n = e / NP, k = e - n * NP;
        const float v = (n < N && k < N) ? A[LAYOUT == 0 ? k * N + n : n * N + k] : 0.f;
        bs[ctc_off<NP>(n, k) / 2] = (unsigned short)(pack_bf16(v, 0.f) & 0xffffu);
    }
    const bool row = tid < N;
    float x[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) x[j] = (row && j == tid) ? 1.f : 0.f;
    for (int k = 0; k < steps; ++k) {
        if (row && !s.aborted) {
#pragma unroll
            for (int g = 0; g < NP / 8; ++g) {
                uint4 q;
                q.x = pack_bf16(x[8 * g + 0], x[8 * g + 1]);
                q.y = pack_bf16(x[8 * g + 2], x[8 * g + 3]);
                q.z = pack_bf16(x[8 * g + 4], x[8 * g + 5]);
                q.w = pack_bf16(x[8 * g + 6], x[8 * g + 7]);
                *reinterpret_cast<uint4*>(smem + ctc_off<NP>(tid, 8 * g)) = q;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        lt_tc_fence_before();
        __syncthreads();
        if (tid == 0 && !s.aborted) {
            lt_tc_fence_after();
#pragma unroll
            for (int kb = 0; kb < NP / 16; ++kb) {
                const unsigned long long da = lt_tc_desc(s.a_u + kb * 256u, 128u, ChainTC<N>::SBO);
                const unsigned long long db = lt_tc_desc(s.b_u + kb * 256u, 128u, ChainTC<N>::SBO);
                ctc_mma_bf16(s.tmem, da, db, ChainTC<N>::IDESC, kb > 0);
            }
            lt_tc_commit(s.bar);
        }
        const bool ok = s.aborted || lt_mbar_wait(s.bar, (unsigned)s.phase, nullptr);
        const bool ab = __syncthreads_or(!ok) != 0;
        if (ab && !s.aborted) {
            s.aborted = true;
            if (tid == 0) atomicAdd(&cj_wait_timeouts, 1u);
        }
        if (s.aborted) continue;
        s.phase ^= 1;
        lt_tc_fence_after();
        if (warp * 32 < N) {   // warps holding a real row read their accumulator lanes
#pragma unroll
            for (int c = 0; c < NP; c += 16) {
                float v[16];
                lt_tmem_ld16(s.tmem + ((unsigned)(warp * 32) << 16) + c, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) x[c + i] = __fmaf_rn(cc, v[i], x[c + i]);
            }
        }
        lt_tc_fence_before();
    }
    if (row && !s.aborted) {
#pragma unroll
        for (int j = 0; j < N; ++j) X[LAYOUT == 0 ? tid * N + j : j * N + tid] = x[j];
    }
    __syncthreads();   // the B operand is rewritten by the next instance
}

template <int N>
__device__ __forceinline__ void chain_tc_teardown(ChainTC<N>& s) {
    // after an expired wait, give the MMAs in flight a bounded second chance
    // to complete before their tensor memory is freed
    if (s.aborted && threadIdx.x == 0) lt_mbar_wait(s.bar, (unsigned)s.phase, nullptr);
    lt_tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        lt_tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(ChainTC<N>::TCOLS)
                     : "memory");
    }
}

// Batched: persistent CTAs take instances blockIdx.x, blockIdx.x + gridDim.x, ...
template <int N, int LAYOUT>
__global__ void __launch_bounds__(128)
update_chain_tc(const float* __restrict__ A, float* __restrict__ X, long long batch, int steps, double c, int ipb) {
    static_assert(N >= 16 && N <= 64, "mapping 7: 16 <= N <= 64");
    extern __shared__ __align__(128) unsigned char cj_smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_slot;
    (void)ipb;   // one instance per CTA at a time
    ChainTC<N> s;
    chain_tc_setup<N>(s, cj_smem, &bar, &tmem_slot);
    const float cc = (float)c;
    for (long long b = blockIdx.x; b < batch; b += gridDim.x)
        chain_tc_instance<N, LAYOUT>(s, cj_smem, A + b * N * N, X + b * N * N, steps, cc);
    chain_tc_teardown<N>(s);
}

// Grouped (a work list of one size N, different T): items {offset, T, 0}
// taken one at a time from the counter.
template <int N>
__global__ void __launch_bounds__(128)
update_chain_grouped_tc(const long long* __restrict__ items, const float* __restrict__ A_pool,
                        float* __restrict__ X_pool, int* __restrict__ counter, long long n_items) {
    static_assert(N >= 16 && N <= 64, "mapping 7: 16 <= N <= 64");
    extern __shared__ __align__(128) unsigned char cj_smem[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_slot;
    __shared__ long long s_item[2];
    ChainTC<N> s;
    chain_tc_setup<N>(s, cj_smem, &bar, &tmem_slot);
    for (;;) {
        if (threadIdx.x == 0) {
            const long long i = atomicAdd(counter, 1);
            s_item[0] = i < n_items ? items[3 * i] : -1;
            s_item[1] = i < n_items ? items[3 * i + 1] : 0;
        }
        __syncthreads();
        const long long off = s_item[0];
        const int steps = (int)s_item[1];
        __syncthreads();
        if (off < 0) break;
        chain_tc_instance<N, 0>(s, cj_smem, A_pool + off, X_pool + off, steps,
                                (float)(1.0 / ((double)N * (double)steps)));
    }
    chain_tc_teardown<N>(s);
}

}  // namespace cj
#endif
