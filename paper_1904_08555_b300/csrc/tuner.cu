// tuner.cu -- autotuner and learned cost model (the paper's future work on
// profiling-guided autotuning of JIT-compiled code, Sec. 6):
//   * cj_candidates: the tile space V(kernel, dtype, N, orders) searched;
//   * cj_autotune:   compile every candidate and time it on the caller's
//                    buffers (exhaustive search; the fallback, and the yardstick
//                    of the model's regret);
//   * cj_featurize:  the cost model's input vector for (request, tile);
//   * cj_mlp_*:      the F -> 64 -> 64 -> 1 ReLU network that predicts the
//                    log run time, with forward, gradient and Adam kernels;
//   * cj_choose_tile / cost-model hook of cj_specialize: argmin of the
//                    predicted time over V.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "cj.h"
#include "cj_internal.h"
#include "kernels/geometry.h"
#include "kernels/mlp.cuh"

#define CJ_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int H = 64;      // hidden width
constexpr int BS = 64;     // samples per block in the gradient kernel

cj_status tfail(cj_status s, const char *msg) {
    cjint::set_last_error(msg);
    return s;
}

int esize(int dtype) { return dtype == CJ_F64 ? 8 : 4; }

// ---------------------------------------------------------------------------
// Candidate tiles
// ---------------------------------------------------------------------------
bool g_fast(int lay) { return lay == 1 || lay == 4; }
bool z_fast(int lay) { return lay == 0 || lay == 2; }

void chain_candidates(const cj_template_args &a, std::vector<std::array<int, 4>> &out) {
    const int n = a.n, es = esize(a.dtype);
    auto ok = [&](int map, int ipb) {
        return cjg::chain_threads(n, map, ipb) <= 1024 && cjg::chain_smem(n, map, ipb, es) <= 200 * 1024;
    };
    if (a.dtype == CJ_BF16) {   // mma.sync panels (mapping 3) and tcgen05 (mapping 7)
        for (int ipb : {1, 2, 4, 8})
            if (ok(3, ipb)) out.push_back({3, ipb, 0, 0});
        out.push_back({7, 1, 0, 0});
        return;
    }
    if (a.dtype == CJ_F64 && n % 8 == 0 && n <= 32)
        for (int ipb : {1, 2, 4, 8})
            if (ok(4, ipb)) out.push_back({4, ipb, 0, 0});
    if (a.dtype == CJ_F32 && n >= 16)   // 4 x 8 register blocks: blocks of 128 to 512 threads
        for (int ipb : {1, 2, 4, 8, 16, 32, 64})
            if (ok(8, ipb) && cjg::chain_threads(n, 8, ipb) >= 128 && cjg::chain_threads(n, 8, ipb) <= 512)
                out.push_back({8, ipb, 0, 0});
    if (a.dtype == CJ_F32 && n >= 8)   // 4 x 4 blocks: from n = 16 on, mapping 8's space covers the large blocks
        for (int ipb : {1, 2, 4, 8, 16, 32})
            if (ok(5, ipb) && cjg::chain_threads(n, 5, ipb) >= 64 && (n < 16 || cjg::chain_threads(n, 5, ipb) <= 256))
                out.push_back({5, ipb, 0, 0});
    if (a.dtype == CJ_F32)
        for (int ipb : {1, 2, 4, 8, 16, 32})
            if (ok(6, ipb) && cjg::chain_threads(n, 6, ipb) >= 64) out.push_back({6, ipb, 0, 0});
    if (n <= 8)
        for (int ipb : {32, 64, 128, 256})
            if (ok(2, ipb)) out.push_back({2, ipb, 0, 0});
    for (int ipb : {2, 4, 8, 16, 32, 64})
        if (ipb * n <= 1024 && ok(1, ipb)) out.push_back({1, ipb, 0, 0});
}

void ltimes_candidates(const cj_template_args &a, std::vector<std::array<int, 4>> &out) {
    const int es = esize(a.dtype);
    const bool gi = g_fast(a.layout_a), go = g_fast(a.layout_b);
    std::vector<int> tgs;
    const int rule = (!gi && !go) ? 1 : ((gi && z_fast(a.layout_b)) || (go && z_fast(a.layout_a))) ? 8 : 32;
    tgs.push_back(rule);
    tgs.push_back(rule == 1 ? 8 : 1);
    auto push = [&](int tg, int ct, int mode, int r, int s, int pipe = 0) {
        if (ct % tg) return;
        int nt;
        if (mode == 1) {
            if (ct % (8 * r)) return;
            nt = ct / (8 * r) * 32;
        } else if (mode == 2) {
            if (ct % 16 || a.d % 8) return;
            nt = ct / 16 * 32;
        } else if (mode == 5) {   // tcgen05 + TMA: r = operand stages, s = converter warps, pipe = TMA boxes
            static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            const int inner = order[a.layout_a][2];
            if (ct != 128 || a.dtype != CJ_F32 || a.m > 128 || (inner == 0 ? 32 : inner == 1 ? tg : ct / tg) % 4) return;
            if (cjg::lt_tc_smem(a.m, a.d, r, tg, ct / tg, a.layout_b, pipe) > 220 * 1024) return;
            out.push_back({tg, ct / tg, 32 * (6 + s), (pipe << 20) | (5 << 16) | (r << 8) | s});
            return;
        } else if (mode == 6) {   // tcgen05 + TMA, operands in TMEM: r = TMEM stages, s = converter warps, pipe = boxes
            static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            const int inner = order[a.layout_a][2];
            const int npa = (cjg::lt_tc_np(a.m) + 31) / 32 * 32;
            if (ct != 128 || a.dtype != CJ_F32 || a.m > 128 || (inner == 0 ? 32 : inner == 1 ? tg : ct / tg) % 4) return;
            if (2 * npa + 64 * r > 512 || cjg::lt_tc_smem(a.m, a.d, 0, tg, ct / tg, a.layout_b, pipe) > 220 * 1024 ||
                cjg::lt_tc_smem(a.m, a.d, 2, tg, ct / tg, a.layout_b) > 220 * 1024)
                return;
            out.push_back({tg, ct / tg, 32 * (6 + s), (pipe << 20) | (6 << 16) | (r << 8) | s});
            return;
        } else if (mode == 4) {   // tcgen05: r = stages, s = producer warps
            if (ct != 128 || a.dtype != CJ_F32 || a.m > 128) return;
            if (cjg::lt_tc_smem(a.m, a.d, r, tg, ct / tg, a.layout_b) > 220 * 1024) return;
            out.push_back({tg, ct / tg, 32 * (5 + s), (4 << 16) | (r << 8) | s});
            return;
        } else if (mode == 3) {
            if (ct % r || (s && (s % 4 || s >= a.m))) return;
            nt = ct / r * (s ? (a.m + s - 1) / s : 1);
            if (nt < 32 || nt > 1024) return;
            if (cjg::lt_direct_smem(a.m, a.d, ct, es, s) > 200 * 1024) return;
            out.push_back({tg, ct / tg, nt, (3 << 16) | (r << 8) | s});
            return;
        } else {
            if (ct % r) return;
            nt = (ct / r) * ((a.m + s - 1) / s);
        }
        if (nt < 32 || nt > 1024) return;
        if (cjg::lt_smem(a.m, s, a.d, ct, es, pipe, mode) > 200 * 1024) return;
        out.push_back({tg, ct / tg, nt, (pipe << 20) | (mode << 16) | (r << 8) | s});
    };
    for (int tg : tgs) {
        if (a.dtype == CJ_F64) {
            if (a.d % 4 == 0)
                for (int ct : {64, 128})
                    for (int r : {1, 2, 4}) push(tg, ct, 1, r, 8);
            push(tg, 64, 0, 1, 9);
            push(tg, 64, 0, 1, 12);
        } else {
            push(tg, 128, 6, 4, 4, 6);          // tcgen05 3xTF32, TMA, operands in TMEM: 6 boxes, 4 stages, 4 converters
            push(tg, 128, 6, 4, 8, 6);          //                                        8 converters
            push(tg, 128, 5, 2, 8, 4);          // tcgen05 3xTF32 fed by TMA: 4 boxes, 2 operand stages
            push(tg, 128, 4, 2, 8);             // tcgen05 3xTF32, register producers: 2 operand stages
            push(tg, 64, 2, 1, 8, 1);           // mma.sync 3xTF32
            push(tg, 64, 0, 2, 12, 1);          // FMA, cp.async double buffer
            push(tg, 256, 3, 2, 0, 0);          // direct loads, all moments per thread
            if (a.m > 12) push(tg, 128, 3, 2, 12, 0);   // direct loads, 12 moments per thread
        }
    }
}

// LPlusTimes runs the LTimes kernel of the swapped problem.
cj_template_args lt_swapped(int k, const cj_template_args &a) {
    if (k != CJ_K_LPLUSTIMES) return a;
    cj_template_args s = a;
    s.m = a.d;
    s.d = a.m;
    s.layout_a = a.layout_b;
    s.layout_b = a.layout_a;
    return s;
}

// ---------------------------------------------------------------------------
// Features
// ---------------------------------------------------------------------------
double lg2(double v) { return std::log2(std::max(v, 1.0)); }
// Axis (0 = d or m, 1 = g, 2 = z) at slot s (0 slowest .. 2 fastest) of storage order lay.
int lt_axis(int lay, int s) {
    static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    return order[((lay % 6) + 6) % 6][s];
}

void featurize(int k, const cj_template_args &a0, int64_t batch, int32_t steps, const int *tile, float *f) {
    std::memset(f, 0, sizeof(float) * CJ_FEATURES);
    const cj_template_args a = lt_swapped(k, a0);
    f[0] = k == CJ_K_UPDATE_CHAIN;
    f[1] = k == CJ_K_LTIMES || k == CJ_K_LPLUSTIMES;
    f[2] = k == CJ_K_UPDATE_CHAIN_GROUPED;
    f[3 + std::min(std::max(a.dtype, 0), 2)] = 1.f;
    const int es = esize(a.dtype);
    double flops, bytes;
    if (k == CJ_K_LTIMES || k == CJ_K_LPLUSTIMES) {
        const double cols = (double)batch;
        flops = 2.0 * a.m * a.d * cols;
        bytes = es * ((double)(a.d + a.m) * cols + a.m * a.d);
        f[6] = lg2(a.m) / 6;
        f[7] = lg2(a.d) / 7;
        // storage orders by their physical shape rather than by name: which
        // axis is fastest and which is in the middle, for `in` (x = d) and for
        // `out` (x = m).  Orders that share a fastest axis share the features
        // that decide coalescing, so unseen pairs of orders relate to seen ones.
        f[8 + lt_axis(a.layout_a, 2)] = 1.f;
        f[11 + lt_axis(a.layout_a, 1)] = 1.f;
        f[14 + lt_axis(a.layout_b, 2)] = 1.f;
        f[17 + lt_axis(a.layout_b, 1)] = 1.f;
        const int mode = (tile[3] >> 16) & 0xf, r = (tile[3] >> 8) & 0xff, s = tile[3] & 0xff;
        // f[2] and f[5] (grouped kernel, bf16) are always 0 for LTimes; here they
        // flag the tcgen05 tiles (modes 4-6) and the TMA-fed ones (modes 5, 6;
        // f[25] tells 6, the tensor-memory operands, apart)
        f[2] = mode >= 4 && mode <= 6;
        f[5] = mode == 5 || mode == 6;
        f[26] = ((tile[3] >> 20) & 0xf) / 8.f;   // cp.async flag, prefetch depth or TMA boxes
        f[20] = lg2(tile[0]) / 5;
        f[21] = lg2(tile[1]) / 7;
        f[22] = lg2(tile[2]) / 10;
        f[23] = r / 8.f;
        f[24] = s / 16.f;
        f[25] = mode / 5.f;
    } else {
        const double n = a.n;
        flops = (double)batch * steps * (2 * n * n * n + 2 * n * n);
        bytes = (double)batch * 2 * n * n * es;
        f[6] = lg2(n) / 6;
        f[7] = n / 64;
        f[8 + (a.layout_a & 1)] = 1.f;
        // the Eigen recurrence's mappings are the chain's thread shapes: 1 = one
        // row per thread (chain mapping 1), 2 = two rows per thread (mapping 6)
        const int map = k == CJ_K_EIGEN_RECURRENCE ? (tile[0] == 2 ? 6 : 1) : tile[0];
        f[20] = map == 1 || map == 6;
        f[21] = map == 2;
        f[22] = map == 4 || map == 5 || map == 8;   // register/tensor blocked panels
        f[19] = map == 5 ? 1.f : map == 8 ? 1.5f : map == 6 ? 0.5f : 0.f;
        f[16] = map == 7;   // tcgen05 tensor cores
        f[23] = lg2(tile[1]) / 8;
        const int threads = cjg::chain_threads(a.n, map, tile[1]);
        f[24] = lg2(threads) / 10;
        f[25] = a.n % 8 == 0;
        f[26] = steps / 128.f;
        // structural consequences of (n, tile) the kernels' code makes:
        // A held in registers, rows of X in shared memory, work wasted on
        // zero padding, resident blocks per SM and waves over the batch
        const bool a_regs = es == 8 ? a.n * a.n <= 64 : a.n * a.n <= 100;
        f[10] = (map == 1 || map == 6) && a_regs;
        f[11] = (map == 1 && a.n > cjg::chain_reg_rows_max(es)) || (map == 6 && a.n > 32);
        const double np = map == 5 ? (a.n + 3) / 4 * 4 : (map == 3 || map == 7) ? (a.n + 15) / 16 * 16 : a.n;
        // mapping 8 pads rows to 4 and columns to 8 and sums over the n real k
        const double work = map == 8 ? (double)((a.n + 3) / 4 * 4) * ((a.n + 7) / 8 * 8) * a.n : np * np * np;
        f[12] = (float)(work / ((double)a.n * a.n * a.n) - 1.0);
        const long smem = k == CJ_K_EIGEN_RECURRENCE ? cjg::eig_smem(a.n, tile[1], es, tile[0])
                                                       : cjg::chain_smem(a.n, map, tile[1], es);
        const double per_sm = std::max(1.0, std::min(2048.0 / threads, 228.0 * 1024 / std::max(smem, 1L)));
        f[13] = (float)(std::min(per_sm, 32.0) / 32.0);
        f[14] = lg2((double)smem) / 18;
        const double blocks = std::ceil((double)batch / tile[1]);
        f[15] = (float)(lg2(blocks / (148.0 * std::floor(per_sm))) / 10);
    }
    f[27] = lg2((double)batch) / 27;
    f[28] = lg2(flops) / 45;
    f[29] = lg2(bytes) / 35;
    f[30] = (float)(std::log2(std::max(flops, 1.0) / std::max(bytes, 1.0)) / 10);
    // whether this is the tile the library's default rule picks for the
    // request: the network learns the rule's corrections rather than the
    // rule itself (a constant input here would only repeat the biases)
    int def[4];
    cjint::default_tile_of(k, a0, def);
    f[31] = std::equal(def, def + 4, tile) ? 1.f : 0.f;
}

cj_status candidates(int k, const cj_template_args &a, std::vector<std::array<int, 4>> &out) {
    out.clear();
    if (k == CJ_K_LTIMES || k == CJ_K_LPLUSTIMES) ltimes_candidates(lt_swapped(k, a), out);
    else if (k == CJ_K_MASS) {
        for (int pipe : {0, 1})   // one group per block (7 sizes); persistent with staged loads (3)
            for (int epb : {1, 2, 4, 8, 16, 32, 64})
                if ((pipe == 0 || epb == 4 || epb == 16 || epb == 64) && cjg::mass_threads(a.n, a.m, epb) <= 1024 &&
                    cjg::mass_smem(a.d, a.n, a.m, epb, esize(a.dtype), pipe) <= 200 * 1024)
                    out.push_back({epb, pipe, 0, 0});
        if (cjg::mass_thread_ok(a.d, a.n, a.m))   // 2-D, one thread per element
            for (int epb : {64, 128, 256}) out.push_back({epb, 2, 0, 0});
    } else if (k == CJ_K_EIGEN_RECURRENCE) {
        for (int map : {1, 2}) {
            if (map == 2 && a.dtype != CJ_F32) continue;
            for (int ipb : {1, 2, 4, 8, 16, 32, 64})
                if (cjg::chain_threads(a.n, map == 2 ? 6 : 1, ipb) <= 1024 &&
                    cjg::eig_smem(a.n, ipb, esize(a.dtype), map) <= 200 * 1024)
                    out.push_back({map, ipb, 0, 0});
        }
    } else chain_candidates(a, out);
    if (out.empty()) return tfail(CJ_ERR_INVALID_ARG, "no candidate tile fits these arguments");
    // the default rule's tile is always searched too (first, if the space
    // above does not hold it), so a tuned choice is never worse than the
    // default on the autotuner's own timings
    std::array<int, 4> def{};
    cjint::default_tile_of(k, a, def.data());
    if (std::find(out.begin(), out.end(), def) == out.end()) out.insert(out.begin(), def);
    return CJ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// MLP object
// ---------------------------------------------------------------------------
struct cj_mlp_s {
    int F = 0, P = 0, step = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    float *partial = nullptr, *partial_loss = nullptr;
    int64_t partial_blocks = 0;
    float *feat = nullptr, *pred = nullptr;   // cost-model query buffers
    std::mutex mu;
};

namespace {

std::mutex g_model_mu;
std::vector<cj_mlp> g_models;   // the installed ensemble (cj_specialize with tile = 0, cj_choose_tile)

uint64_t splitmix(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

size_t grad_smem(int F, int P) {
    return sizeof(float) * ((size_t)((P + 3) & ~3) + (size_t)BS * F + 3u * BS * H + 2u * BS);
}

cj_status ensure_partials(cj_mlp m, int64_t blocks) {
    if (blocks <= m->partial_blocks) return CJ_OK;
    if (m->partial) cudaFree(m->partial);
    if (m->partial_loss) cudaFree(m->partial_loss);
    m->partial = m->partial_loss = nullptr;
    if (cudaMalloc(&m->partial, sizeof(float) * blocks * m->P) != cudaSuccess ||
        cudaMalloc(&m->partial_loss, sizeof(float) * blocks) != cudaSuccess) {
        m->partial_blocks = 0;
        return tfail(CJ_ERR_OOM, "cost model: could not allocate gradient partials");
    }
    m->partial_blocks = blocks;
    return CJ_OK;
}

cj_status grad_pass(cj_mlp m, const float *X, const float *t, int64_t B, cudaStream_t st, int apply, float lr,
                    float *grad_out, float *loss_out) {
    const int64_t blocks = (B + BS - 1) / BS;
    cj_status rc = ensure_partials(m, blocks);
    if (rc != CJ_OK) return rc;
    const size_t smem = grad_smem(m->F, m->P);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(cj::mlp_grad_partial<H, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    });
    cj::mlp_grad_partial<H, BS><<<(unsigned)blocks, BS, smem, st>>>(m->theta, X, t, m->F, B, m->partial,
                                                                      m->partial_loss);
    if (apply) m->step++;
    cj::mlp_reduce_adam<<<(m->P + 255) / 256, 256, 0, st>>>(m->partial, m->partial_loss, (int)blocks, m->P, m->theta,
                                                           m->m, m->v, grad_out, loss_out, B, m->step, lr, 0.9f,
                                                           0.999f, 1e-8f, apply);
    if (cudaGetLastError() != cudaSuccess) return tfail(CJ_ERR_CUDA, "cost model: gradient launch failed");
    return CJ_OK;
}

cj_status forward(cj_mlp m, const float *X, int64_t B, float *y, cudaStream_t st) {
    if (B == 0) return CJ_OK;
    const size_t smem = sizeof(float) * m->P;
    cj::mlp_forward<H><<<(unsigned)((B + 127) / 128), 128, smem, st>>>(m->theta, X, y, m->F, B);
    if (cudaGetLastError() != cudaSuccess) return tfail(CJ_ERR_CUDA, "cost model: forward launch failed");
    return CJ_OK;
}

// Predicted log run time of every candidate; returns the argmin.
// Choose a tile for a request: the networks' mean predicted log time over the
// candidates, lowest first, except that the default rule's tile is kept
// unless another candidate is predicted faster by more than kKeepDefault.
cj_status model_choose(const std::vector<cj_mlp> &models, int k, const cj_template_args &a, int64_t batch,
                       int32_t steps, int *tile_out, float *pred_out) {
    std::vector<std::array<int, 4>> cand;
    cj_status rc = candidates(k, a, cand);
    if (rc != CJ_OK) return rc;
    if (cand.size() > 256) return tfail(CJ_ERR_INVALID_ARG, "too many candidates");
    std::vector<float> feat(cand.size() * CJ_FEATURES), pred(cand.size(), 0.f), one(cand.size());
    for (size_t i = 0; i < cand.size(); ++i) featurize(k, a, batch, steps, cand[i].data(), &feat[i * CJ_FEATURES]);
    for (cj_mlp m : models) {
        if (m->F != CJ_FEATURES) return tfail(CJ_ERR_INVALID_ARG, "cost model must have CJ_FEATURES inputs");
        std::lock_guard<std::mutex> lk(m->mu);
        if (!m->feat) {
            if (cudaMalloc(&m->feat, sizeof(float) * 256 * CJ_FEATURES) != cudaSuccess ||
                cudaMalloc(&m->pred, sizeof(float) * 256) != cudaSuccess)
                return tfail(CJ_ERR_OOM, "cost model: query buffers");
        }
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return tfail(CJ_ERR_CUDA, "cost model: stream");
        cudaMemcpyAsync(m->feat, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, st);
        rc = forward(m, m->feat, (int64_t)cand.size(), m->pred, st);
        if (rc == CJ_OK) cudaMemcpyAsync(one.data(), m->pred, sizeof(float) * one.size(), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (rc != CJ_OK) return rc;
        if (e != cudaSuccess) return tfail(CJ_ERR_CUDA, "cost model: query failed");
        for (size_t i = 0; i < pred.size(); ++i) pred[i] += one[i] / (float)models.size();
    }
    size_t best = std::min_element(pred.begin(), pred.end()) - pred.begin();
    // A gain the networks cannot tell from timing noise and the spread of
    // sizes they were not trained on is not worth leaving the rule for.
    std::array<int, 4> def{};
    cjint::default_tile_of(k, a, def.data());
    const size_t di = std::find(cand.begin(), cand.end(), def) - cand.begin();
    constexpr float kKeepDefault = 0.0953102f;   // log(1.10): predicted 10% faster
    if (di < cand.size() && pred[di] - pred[best] <= kKeepDefault) best = di;
    std::memcpy(tile_out, cand[best].data(), sizeof(int) * 4);
    if (pred_out) *pred_out = pred[best];
    return CJ_OK;
}

}  // namespace

namespace cjint {
// Hook used by cj_specialize for tile = {0,0,0,0} when the config enables
// the cost model and a model is installed.  Hints: chain batch 2^22/n^2
// instances with T = 64, LTimes 2^21 columns.
bool cost_model_tile(int k, const cj_template_args &a, int *tile_out) {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (g_models.empty()) return false;
    const int64_t batch = k == CJ_K_LTIMES ? (int64_t)1 << 21 : std::max<int64_t>(1, ((int64_t)1 << 22) / (a.n * a.n));
    return model_choose(g_models, k, a, batch, 64, tile_out, nullptr) == CJ_OK;
}
}  // namespace cjint

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
CJ_API cj_status cj_candidates(cj_kernel_id k, const cj_template_args *a, int32_t *tiles, int32_t cap,
                               int32_t *count) {
    if (!a || !count || (cap > 0 && !tiles)) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    if (a->dtype == CJ_BF16 && k != CJ_K_UPDATE_CHAIN && k != CJ_K_UPDATE_CHAIN_GROUPED)
        return tfail(CJ_ERR_INVALID_ARG, "bf16 candidates exist for the update chain only");
    if (a->dtype == CJ_BF16 && a->n < 16) return tfail(CJ_ERR_INVALID_ARG, "bf16 update chains need n >= 16");
    std::vector<std::array<int, 4>> cand;
    cj_status rc = candidates((int)k, *a, cand);
    if (rc != CJ_OK) return rc;
    *count = (int32_t)cand.size();
    for (int i = 0; i < std::min<int>(cap, (int)cand.size()); ++i) std::memcpy(tiles + 4 * i, cand[i].data(), 16);
    return CJ_OK;
}

CJ_API cj_status cj_featurize(cj_kernel_id k, const cj_template_args *a, int64_t batch, int32_t steps,
                              const int32_t tile[4], float *out) {
    if (!a || !tile || !out || batch < 0) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    if (k == CJ_K_MASS) return tfail(CJ_ERR_INVALID_ARG, "the cost model has no features for the mass operator");
    featurize((int)k, *a, batch, steps, tile, out);
    return CJ_OK;
}

CJ_API cj_status cj_autotune(cj_kernel_id k, const cj_template_args *a, void *const *launch_args, int64_t batch,
                             void *cuda_stream, int32_t reps, int32_t best_tile[4], float *times_ms, int32_t cap,
                             int32_t *count) {
    if (!a || !launch_args || !best_tile || !count || reps < 1) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    std::vector<std::array<int, 4>> cand;
    cj_status rc = candidates((int)k, *a, cand);
    if (rc != CJ_OK) return rc;
    // compile everything first (queued in async mode), then time
    std::vector<cj_handle> hs(cand.size());
    for (size_t i = 0; i < cand.size(); ++i) {
        cj_template_args r = *a;
        std::memcpy(r.tile, cand[i].data(), 16);
        r.flags = (r.flags & ~(uint32_t)CJ_FLAG_GENERIC) | CJ_FLAG_NO_AOT;
        rc = cj_specialize(k, &r, &hs[i]);
        if (rc != CJ_OK && rc != CJ_ERR_COMPILE) return rc;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    *count = (int32_t)cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
        float ms = INFINITY;
        if (cj_specialize_wait(hs[i], -1) == CJ_OK) {
            rc = cj_launch(hs[i], launch_args, batch, cuda_stream);   // warm-up
            if (rc != CJ_OK) break;
            std::vector<float> t(reps);
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, st);
                cj_launch(hs[i], launch_args, batch, cuda_stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&t[r], e0, e1);
            }
            std::sort(t.begin(), t.end());
            ms = t[reps / 2];
        }
        if (times_ms && (int)i < cap) times_ms[i] = ms;
        if (ms < best) {
            best = ms;
            std::memcpy(best_tile, cand[i].data(), 16);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CJ_OK) return rc;
    if (best >= 1e30f) return tfail(CJ_ERR_COMPILE, "no candidate compiled");
    return CJ_OK;
}

CJ_API cj_status cj_mlp_create(int32_t in_features, uint64_t seed, cj_mlp *out) {
    if (!out || in_features < 1 || in_features > 64) return tfail(CJ_ERR_INVALID_ARG, "in_features must be 1..64");
    auto *m = new cj_mlp_s();
    m->F = in_features;
    m->P = cj::MlpLayout<H>{in_features}.count();
    const size_t bytes = sizeof(float) * m->P;
    if (cudaMalloc(&m->theta, bytes) != cudaSuccess || cudaMalloc(&m->m, bytes) != cudaSuccess ||
        cudaMalloc(&m->v, bytes) != cudaSuccess || cudaMalloc(&m->grad, bytes) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
        cj_mlp_destroy(m);
        return tfail(CJ_ERR_OOM, "cost model: parameter allocation failed");
    }
    // uniform(-s, s) weights with s = sqrt(3 / fan_in) (unit-variance inputs keep unit variance), zero biases
    std::vector<float> h(m->P, 0.f);
    const cj::MlpLayout<H> L{in_features};
    auto fill = [&](int off, int cnt, int fan_in, uint64_t stream) {
        const double s = std::sqrt(3.0 / fan_in);
        for (int i = 0; i < cnt; ++i) {
            const double u = (double)(splitmix(seed + stream, (uint64_t)i) >> 11) * 0x1.0p-53;
            h[off + i] = (float)((2 * u - 1) * s);
        }
    };
    fill(L.w1(), H * in_features, in_features, 1);
    fill(L.w2(), H * H, H, 2);
    fill(L.w3(), H, H, 3);
    cj_status rc = cj_mlp_set_params(m, h.data(), m->P);
    if (rc != CJ_OK) {
        cj_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return CJ_OK;
}

CJ_API cj_status cj_mlp_set_params(cj_mlp m, const float *host, int64_t count) {
    if (!m || !host || count != m->P) return tfail(CJ_ERR_INVALID_ARG, "parameter count mismatch");
    if (cudaMemcpy(m->theta, host, sizeof(float) * m->P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, sizeof(float) * m->P) != cudaSuccess ||
        cudaMemset(m->v, 0, sizeof(float) * m->P) != cudaSuccess)
        return tfail(CJ_ERR_CUDA, "cost model: parameter upload failed");
    m->step = 0;
    return CJ_OK;
}

CJ_API cj_status cj_mlp_get_params(cj_mlp m, float *host, int64_t cap, int64_t *count) {
    if (!m || !count) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    *count = m->P;
    if (host && cap >= m->P &&
        cudaMemcpy(host, m->theta, sizeof(float) * m->P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return tfail(CJ_ERR_CUDA, "cost model: parameter download failed");
    return CJ_OK;
}

CJ_API cj_status cj_mlp_forward(cj_mlp m, const float *X, int64_t B, float *y, void *cuda_stream) {
    if (!m || B < 0 || (B > 0 && (!X || !y))) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    return forward(m, X, B, y, reinterpret_cast<cudaStream_t>(cuda_stream));
}

CJ_API cj_status cj_mlp_grad(cj_mlp m, const float *X, const float *t, int64_t B, float *grad, float *loss,
                             void *cuda_stream) {
    if (!m || B < 1 || !X || !t || !grad) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    return grad_pass(m, X, t, B, reinterpret_cast<cudaStream_t>(cuda_stream), 0, 0.f, grad, loss);
}

CJ_API cj_status cj_mlp_train_step(cj_mlp m, const float *X, const float *t, int64_t B, float lr, float *loss,
                                   void *cuda_stream) {
    if (!m || B < 1 || !X || !t || lr <= 0.f) return tfail(CJ_ERR_INVALID_ARG, "bad argument");
    return grad_pass(m, X, t, B, reinterpret_cast<cudaStream_t>(cuda_stream), 1, lr, m->grad, loss);
}

CJ_API cj_status cj_mlp_destroy(cj_mlp m) {
    if (!m) return tfail(CJ_ERR_INVALID_ARG, "null model");
    {
        std::lock_guard<std::mutex> lk(g_model_mu);
        if (std::find(g_models.begin(), g_models.end(), m) != g_models.end()) g_models.clear();
    }
    for (float *p : {m->theta, m->m, m->v, m->grad, m->loss, m->partial, m->partial_loss, m->feat, m->pred})
        if (p) cudaFree(p);
    delete m;
    return CJ_OK;
}

CJ_API cj_status cj_cost_model_use_ensemble(const cj_mlp *m, int32_t count) {
    if (count < 0 || (count > 0 && !m)) return tfail(CJ_ERR_INVALID_ARG, "null models or negative count");
    for (int32_t i = 0; i < count; ++i)
        if (!m[i] || m[i]->F != CJ_FEATURES) return tfail(CJ_ERR_INVALID_ARG, "cost model must have CJ_FEATURES inputs");
    std::lock_guard<std::mutex> lk(g_model_mu);
    g_models.assign(m, m + count);
    return CJ_OK;
}

CJ_API cj_status cj_cost_model_use(cj_mlp m) { return cj_cost_model_use_ensemble(m ? &m : nullptr, m ? 1 : 0); }

CJ_API cj_status cj_choose_tile(cj_kernel_id k, const cj_template_args *a, int64_t batch, int32_t steps,
                                int32_t tile_out[4], float *predicted) {
    if (!a || !tile_out || batch < 1) return tfail(CJ_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (g_models.empty()) return tfail(CJ_ERR_INVALID_ARG, "no cost model installed (cj_cost_model_use)");
    return model_choose(g_models, (int)k, *a, batch, steps, tile_out, predicted);
}
