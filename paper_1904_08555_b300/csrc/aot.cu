// aot.cu -- kernels compiled ahead of time by nvcc for sm_103a: the generic
// runtime-N kernels (the stand-ins while a specialization compiles, and the
// fallback if it fails) and the explicit specializations n in {4, 8, 16, 32}
// of the update chain.  Explicit specializations are used instead of JIT
// compiling the same instantiation (Sec. 2).
#include "cj_internal.h"
#include "kernels/ltimes.cuh"
#include "kernels/mass.cuh"
#include "kernels/update_chain.cuh"

using namespace cjint;

#define CJ_AOT_CHAIN(T, DT, N, L)                                                                 \
    {K_CHAIN, DT, N, L, {chain_default_map(N, DT), chain_default_ipb(N, DT), 0, 0},              \
     (const void *)&cj::update_chain<T, N, L, chain_default_map(N, DT), chain_default_ipb(N, DT)>}

#define CJ_AOT_CHAIN_SIZES(T, DT, L) \
    CJ_AOT_CHAIN(T, DT, 4, L), CJ_AOT_CHAIN(T, DT, 8, L), CJ_AOT_CHAIN(T, DT, 16, L), CJ_AOT_CHAIN(T, DT, 32, L)

static const AotKernel kAotTable[] = {
    CJ_AOT_CHAIN_SIZES(double, D_F64, 0), CJ_AOT_CHAIN_SIZES(double, D_F64, 1),
    CJ_AOT_CHAIN_SIZES(float, D_F32, 0),  CJ_AOT_CHAIN_SIZES(float, D_F32, 1),
};

static const GenericKernels kGeneric = {
    {(const void *)&cj::update_chain_generic<double>, (const void *)&cj::update_chain_generic<float>},
    {(const void *)&cj::ltimes_generic<double>, (const void *)&cj::ltimes_generic<float>},
    {(const void *)&cj::update_chain_grouped_generic<double>,
     (const void *)&cj::update_chain_grouped_generic<float>},
    {(const void *)&cj::eigen_recurrence_generic<double>, (const void *)&cj::eigen_recurrence_generic<float>},
    {(const void *)&cj::mass_apply_generic<double>, (const void *)&cj::mass_apply_generic<float>},
};

// Roofline denominator: 8 independent FMA chains per thread and nothing else
// in the loop.  The store is never taken (the chains converge near
// b / (1 - a)), it only keeps the arithmetic alive.
__device__ double cj_peak_sink;

template <class T>
__global__ void __launch_bounds__(256) peak_fma(int iters, T a, T b) {
    T acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = cj::fmaT(acc[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += acc[i];
    if (s == (T)-123456.0) cj_peak_sink = (double)s;
}

// FP64 tensor-core rate: 8 independent mma.sync m8n8k4 accumulators per
// warp (512 FMA per instruction); the same never-taken store.
template <class T>
__global__ void __launch_bounds__(256) peak_dmma(int iters, T a0, T b0) {
    double c[8][2];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i][0] = threadIdx.x * 1e-3;
        c[i][1] = i * 1e-3;
    }
    const double a = a0 + threadIdx.x * 1e-9, b = b0;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[i][0]), "+d"(c[i][1])
                         : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += c[i][0] + c[i][1];
    if (s == -123456.0) cj_peak_sink = s;
}

namespace cjint {
const void *peak_fma_kernel(int dtype) {
    return dtype == D_F64 ? (const void *)&peak_fma<double> : (const void *)&peak_fma<float>;
}
const void *peak_dmma_kernel() { return (const void *)&peak_dmma<double>; }
const AotKernel *aot_table(int *count) {
    *count = (int)(sizeof(kAotTable) / sizeof(kAotTable[0]));
    return kAotTable;
}
const GenericKernels &generic_kernels() { return kGeneric; }
}  // namespace cjint
