// noalloc.cu -- cj_update_chain_uneven_noalloc: the uneven-batch update chain
// for callers that must not allocate device memory.
//
// Who needs it: code that runs under a device-memory budget owned by someone
// else (a framework's caching allocator, an arena in an embedded or real-time
// deployment) may not call cudaMalloc at all, and code on a latency-critical
// path cannot afford cudaMalloc/cudaFree, which may synchronize the device.
// The grouped plan (cj_group_plan_*) keeps its work lists and counters in
// memory it allocates; this entry point keeps them instead in one fixed
// file-scope __device__ array that the CUDA runtime places in every device's
// context when the library's kernels are loaded, and that stays there until
// the process exits.
//
// The work per instance is the same as the grouped plan's generic path:
// instances are grouped by n, each group's items are ordered by T
// descending, and a persistent kernel per group pulls chunks of items from a
// counter.  Groups run one after another on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "cj.h"
#include "cj_internal.h"
#include "kernels/update_chain.cuh"

namespace {

constexpr size_t kItemBytes = (size_t)CJ_NOALLOC_MAX_INSTANCES * 3 * sizeof(long long);
constexpr size_t kCounterBytes = 256;   // one int32 per n in 1..64
constexpr size_t kScratchBytes = kItemBytes + kCounterBytes;
static_assert(kItemBytes % 256 == 0, "counters must stay 256-byte aligned");

// The scratch array.  In host code this name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char cj_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};   // device address of cj_noalloc_scratch, per device


// Same chunked persistent loop as the generic grouped kernel, with the work
// list and the counter taken from the scratch array.
template <class T>
__global__ void __launch_bounds__(128)
chain_uneven_noalloc(const long long *__restrict__ items, int *__restrict__ counter,
                     const T *__restrict__ A_pool, T *__restrict__ X_pool, long long n_items, int n, int ipb) {
    extern __shared__ __align__(16) unsigned char cj_smem[];
    __shared__ long long s_off[128];
    __shared__ int s_steps[128];
    __shared__ int s_chunk;
    T *sA = reinterpret_cast<T *>(cj_smem);
    const int nn = n * n;
    const int P = cjg::row_pitch(nn, (int)sizeof(T));
    const int XP = cjg::xrow_pitch(n);
    const int nthreads = blockDim.x;
    const int tid = threadIdx.x;
    T *xs = sA + ipb * P + tid * XP;
    T *ps = sA + ipb * P + nthreads * XP + tid * XP;
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
            cj::generic_row_chain<T>(sA + inst * P, xs, ps, n, i, steps, (T)(1.0 / ((double)n * (double)steps)));
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

cj_status na_fail(cj_status s, const std::string &msg) {
    cjint::set_last_error(msg);   // reported by cj_last_error()
    return s;
}

// Once per device, with that device current: the device address of the
// scratch array.
cj_status scratch_for_current_device(int *dev_out, void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return na_fail(CJ_ERR_NO_DEVICE, "cj_update_chain_uneven_noalloc: no current CUDA device");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, cj_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(CJ_ERR_CUDA, std::string("cj_update_chain_uneven_noalloc: cudaGetSymbolAddress failed: ") +
                                            cudaGetErrorString(e));
        const void *k64 = (const void *)&chain_uneven_noalloc<double>;
        const void *k32 = (const void *)&chain_uneven_noalloc<float>;
        int optin = 0;
        cudaFuncAttributes fa64{}, fa32{};
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa64, k64)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa32, k32)) != cudaSuccess)
            return na_fail(CJ_ERR_CUDA, std::string("cj_update_chain_uneven_noalloc: reading the device or kernel "
                                                    "attributes failed: ") + cudaGetErrorString(e));
        if (cudaFuncSetAttribute(k64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa64.sharedSizeBytes) != cudaSuccess ||
            cudaFuncSetAttribute(k32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa32.sharedSizeBytes) != cudaSuccess)
            return na_fail(CJ_ERR_CUDA, "cj_update_chain_uneven_noalloc: could not set the shared-memory limit");
        g_scratch[dev] = p;
    }
    *dev_out = dev;
    *out = g_scratch[dev];
    return CJ_OK;
}

template <class T>
cj_status run(const std::vector<long long> &items, const std::vector<int> &group_n,
              const std::vector<long long> &group_first, const std::vector<long long> &group_count, int dev,
              void *scratch, const void *A_pool, void *X_pool, cudaStream_t st) {
    auto *d_items = reinterpret_cast<long long *>(scratch);
    auto *d_counters = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(scratch) + kItemBytes);
    // The array keeps the previous call's contents: the counters must start at zero.
    if (cudaMemsetAsync(d_counters, 0, kCounterBytes, st) != cudaSuccess)
        return na_fail(CJ_ERR_CUDA, "cj_update_chain_uneven_noalloc: counter reset failed");
    if (!items.empty() && cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(long long),
                                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        return na_fail(CJ_ERR_CUDA, "cj_update_chain_uneven_noalloc: work-list upload failed");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int es = (int)sizeof(T);
    for (size_t g = 0; g < group_n.size(); ++g) {
        const int n = group_n[g];
        const int ipb = std::max(1, 128 / n);
        const int threads = ((ipb * n + 31) / 32) * 32;
        const size_t smem = (size_t)cjg::chain_generic_smem(n, ipb, threads, es);
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_uneven_noalloc<T>, threads, smem);
        const long long chunks = (group_count[g] + ipb - 1) / ipb;
        const unsigned grid = (unsigned)std::min<long long>(chunks, (long long)sms * std::max(1, per_sm));
        chain_uneven_noalloc<T><<<grid, threads, smem, st>>>(d_items + 3 * group_first[g], d_counters + (n - 1),
                                                             static_cast<const T *>(A_pool), static_cast<T *>(X_pool),
                                                             group_count[g], n, ipb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return na_fail(CJ_ERR_CUDA, std::string("cj_update_chain_uneven_noalloc: launch failed: ") +
                                            cudaGetErrorString(e));
    }
    return CJ_OK;
}

}  // namespace

// Forget the per-device set-up (called by cj_shutdown): after a
// cudaDeviceReset the array's address and the kernels' attributes belong to a
// context that no longer exists, so the next call must look them up again.
void cjint::noalloc_forget() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_scratch) p = nullptr;
}

extern "C" __attribute__((visibility("default"))) cj_status
cj_update_chain_uneven_noalloc(int32_t dtype, int64_t count, const int32_t *n, const int32_t *steps,
                               const void *A_pool, void *X_pool, void *cuda_stream) {
    if (dtype != CJ_F64 && dtype != CJ_F32)
        return na_fail(CJ_ERR_INVALID_ARG, "cj_update_chain_uneven_noalloc: dtype must be CJ_F64 or CJ_F32");
    if (count < 0 || (count > 0 && (!n || !steps || !A_pool || !X_pool)))
        return na_fail(CJ_ERR_INVALID_ARG, "cj_update_chain_uneven_noalloc: null argument or negative count");
    if (count > CJ_NOALLOC_MAX_INSTANCES)
        return na_fail(CJ_ERR_INVALID_ARG, "cj_update_chain_uneven_noalloc: " + std::to_string(count) +
                                               " instances exceed the fixed scratch limit of " +
                                               std::to_string(CJ_NOALLOC_MAX_INSTANCES) + " per call");
    for (int64_t k = 0; k < count; ++k)
        if (n[k] < 1 || n[k] > 64 || steps[k] < 1)
            return na_fail(CJ_ERR_INVALID_ARG, "cj_update_chain_uneven_noalloc: instance " + std::to_string(k) +
                                                   " needs 1 <= n <= 64 and T >= 1");
    int dev = -1;
    void *scratch = nullptr;
    cj_status rc = scratch_for_current_device(&dev, &scratch);
    if (rc != CJ_OK) return rc;
    if (count == 0) return CJ_OK;
    // Host-side grouping (host memory only): offsets are the exclusive prefix
    // sums of n^2; items of one n are ordered by T descending.
    std::vector<long long> off(count);
    long long acc = 0;
    for (int64_t k = 0; k < count; ++k) {
        off[k] = acc;
        acc += (long long)n[k] * n[k];
    }
    std::vector<std::vector<int64_t>> by_n(65);
    for (int64_t k = 0; k < count; ++k) by_n[n[k]].push_back(k);
    std::vector<long long> items;
    items.reserve(3 * (size_t)count);
    std::vector<int> group_n;
    std::vector<long long> group_first, group_count;
    for (int nn = 64; nn >= 1; --nn) {
        auto &v = by_n[nn];
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [&](int64_t x, int64_t y) { return steps[x] > steps[y]; });
        group_n.push_back(nn);
        group_first.push_back((long long)items.size() / 3);
        group_count.push_back((long long)v.size());
        for (int64_t k : v) {
            items.push_back(off[k]);
            items.push_back(steps[k]);
            items.push_back(0);
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    return dtype == CJ_F64 ? run<double>(items, group_n, group_first, group_count, dev, scratch, A_pool, X_pool, st)
                           : run<float>(items, group_n, group_first, group_count, dev, scratch, A_pool, X_pool, st);
}
