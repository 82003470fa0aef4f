// cj_internal.h -- declarations shared by the host library (cj.cpp) and the
// ahead-of-time kernel unit (aot.cu).  Not part of the public ABI.
#ifndef CJ_INTERNAL_H
#define CJ_INTERNAL_H

#include <string>

#include "cj.h"

namespace cjint {

enum { K_CHAIN = 1, K_LTIMES = 2, K_GROUPED = 3 };
enum { D_F64 = 0, D_F32 = 1, D_BF16 = 2 };

// Default tile rule of the update chain kernels (documented in cj.h).
// FP64 tensor cores (mapping 4) are a candidate only: on B300 mma.sync f64
// issues on the same FP64 pipe as DFMA and is not faster (measured).
constexpr bool chain_dmma_ok(int n, int dtype) { return dtype == D_F64 && n % 8 == 0 && n <= 32; }
// FP32 n >= 9: two rows per thread (mapping 6), 128 / ceil(n / 2) instances.
// f32 n >= 32: 4 x 8 register blocks (mapping 8), about 128 threads per
// block (t = ceil(n / 4) ceil(n / 8) threads per instance).
constexpr int chain_default_map(int n, int dtype) {
    return dtype == D_BF16 ? 3 : n <= 4 ? 2 : (dtype == D_F32 && n >= 32) ? 8 : (dtype == D_F32 && n >= 9) ? 6 : 1;
}
constexpr int chain_m8_tpi(int n) { return (n + 3) / 4 * ((n + 7) / 8); }
constexpr int chain_default_ipb(int n, int dtype) {
    return dtype == D_BF16 ? (128 / ((n + 15) / 16 * 16) > 1 ? 128 / ((n + 15) / 16 * 16) : 1)
         : n <= 4 ? 128
         : (dtype == D_F32 && n >= 32) ? ((128 + chain_m8_tpi(n) / 2) / chain_m8_tpi(n) > 1
                                              ? (128 + chain_m8_tpi(n) / 2) / chain_m8_tpi(n) : 1)
         : (dtype == D_F32 && n >= 9) ? (128 / ((n + 1) / 2) > 1 ? 128 / ((n + 1) / 2) : 1)
         : n <= 32 ? 256 / n : (128 / n > 1 ? 128 / n : 1);
}

struct AotKernel {
    int kernel, dtype, n, layout;
    int tile[4];
    const void *fn;   // host stub of the __global__ function
};

// Explicit specializations compiled by nvcc (update chain, f64/f32,
// n in {4, 8, 16, 32}, layouts 0 and 1, default tile).
const AotKernel *aot_table(int *count);

// Generic kernels, indexed by dtype (0 f64, 1 f32).
struct GenericKernels {
    const void *chain[2];
    const void *ltimes[2];
    const void *grouped[2];
    const void *eigen[2];
    const void *mass[2];
};
const GenericKernels &generic_kernels();

// FMA-throughput kernel (roofline denominator), indexed by dtype (0 f64, 1 f32):
// kernel(int iters, T a, T b), 256 threads per block, 8 chains per thread.
const void *peak_fma_kernel(int dtype);
// FP64 tensor-core (mma.sync m8n8k4) rate kernel: kernel(int iters, double a, double b).
const void *peak_dmma_kernel();

// Cost-model tile choice for a request with tile = 0 (tuner.cu); false if no
// model is installed or the query failed.
bool cost_model_tile(int k, const cj_template_args &a, int *tile_out);

// The tile the library's default rule picks for request a of kernel k (the
// rule documented in cj.h; no cost model).
void default_tile_of(int k, const cj_template_args &a, int tile_out[4]);

// Drop the allocation-free entry point's per-device set-up (noalloc.cu).
void noalloc_forget();

// Set the thread-local message returned by cj_last_error (used by the
// allocation-free entry point in noalloc.cu).
void set_last_error(const char *msg);
inline void set_last_error(const std::string &msg) { set_last_error(msg.c_str()); }

}  // namespace cjint
#endif
