// cj.cpp -- host side of libcj: the C ABI of include/cj.h, the program-global
// instantiation cache, the NVRTC specializer with its background compile
// threads, the generic / AoT / JIT dispatch and the grouped-plan scheduler.
//
// The runtime follows the paper's Algorithm 1 (Sec. 4) in its CUDA form:
// look the instantiation up in a global cache guarded by a mutex; on a miss,
// instantiate the template from source embedded in this binary (never from a
// file), compile it for the device's architecture and keep the result in the
// cache.  On B300 the device compiler is NVRTC producing sm_103a CUBIN, which
// is loaded with cuLibraryLoadData (the paper built PTX and a fatbin by hand,
// Sec. 4.1).  Unlike the paper, a miss does not block the caller: launches
// use the generic runtime-N kernel until the specialization is ready.
#include "cj.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cj_internal.h"
#include "kernels/geometry.h"

// Kernel template sources, embedded at build time (generated from kernels/).
#include "generated/embedded_sources.inc"

#define CJ_API extern "C" __attribute__((visibility("default")))

namespace {

using clk = std::chrono::steady_clock;

thread_local std::string t_err;

cj_status fail(cj_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

// ---------------------------------------------------------------------------
// Driver API entry points, fetched through the runtime so that the library
// loads on machines without a driver (compile-only use, CPU tests).
// ---------------------------------------------------------------------------
struct Driver {
    CUresult (*LibraryLoadData)(CUlibrary *, const void *, CUjit_option *, void **, unsigned int,
                                CUlibraryOption *, void **, unsigned int) = nullptr;
    CUresult (*LibraryGetKernel)(CUkernel *, CUlibrary, const char *) = nullptr;
    CUresult (*LibraryUnload)(CUlibrary) = nullptr;
    CUresult (*LibraryGetGlobal)(CUdeviceptr *, size_t *, CUlibrary, const char *) = nullptr;
    CUresult (*KernelGetFunction)(CUfunction *, CUkernel) = nullptr;
    CUresult (*FuncSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
    CUresult (*FuncGetAttribute)(int *, CUfunction_attribute, CUfunction) = nullptr;
    CUresult (*LaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                             unsigned, CUstream, void **, void **) = nullptr;
    CUresult (*OccupancyMaxActiveBlocksPerMultiprocessor)(int *, CUfunction, int, size_t) = nullptr;
    CUresult (*GetErrorString)(CUresult, const char **) = nullptr;
    CUresult (*TensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                     const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                     CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                     CUtensorMapFloatOOBfill) = nullptr;
} drv;

template <class F>
bool entry(const char *name, F &fp) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fp = reinterpret_cast<F>(p);
    return true;
}

bool load_driver() {
    return entry("cuLibraryLoadData", drv.LibraryLoadData) && entry("cuLibraryGetKernel", drv.LibraryGetKernel) &&
           entry("cuLibraryUnload", drv.LibraryUnload) && entry("cuLibraryGetGlobal", drv.LibraryGetGlobal) &&
           entry("cuKernelGetFunction", drv.KernelGetFunction) &&
           entry("cuFuncSetAttribute", drv.FuncSetAttribute) && entry("cuFuncGetAttribute", drv.FuncGetAttribute) &&
           entry("cuLaunchKernel", drv.LaunchKernel) &&
           entry("cuOccupancyMaxActiveBlocksPerMultiprocessor", drv.OccupancyMaxActiveBlocksPerMultiprocessor) &&
           entry("cuGetErrorString", drv.GetErrorString) && entry("cuTensorMapEncodeTiled", drv.TensorMapEncodeTiled);
}

const char *cu_str(CUresult r) {
    const char *s = nullptr;
    if (drv.GetErrorString) drv.GetErrorString(r, &s);
    return s ? s : "unknown CUDA driver error";
}

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
enum { ST_PENDING = 0, ST_READY = 1, ST_FAILED = 2, ST_GENERIC_ONLY = 3 };
enum { V_GENERIC = 0, V_AOT = 1, V_JIT = 2 };
constexpr uint32_t kKeyFlags =
    CJ_FLAG_GENERIC | CJ_FLAG_NO_AOT | CJ_FLAG_INJECT_COMPILE_ERROR | CJ_FLAG_INJECT_WAIT_TIMEOUT;

// Everything a launch needs; immutable once published through Handle::impl.
struct Impl {
    CUfunction fn = nullptr;
    int variant = V_GENERIC;
    int threads = 0;
    size_t smem = 0;
    int ipb = 0;            // update chain / grouped: instances per block or chunk
    int blocks_per_sm = 1;  // persistent kernels (LTimes specialized, grouped)
    // LTimes mode 5 only: the mode-4 instantiation of the same tile, launched
    // when `in` admits no TMA tensor map (see launch_ltimes_tc)
    CUfunction fn2 = nullptr;
    int threads2 = 0, blocks2 = 1;
    size_t smem2 = 0;
};

}  // namespace

struct cj_handle_s {
    int kernel = 0;
    cj_template_args a{};   // normalised request, tile resolved
    unsigned char key[32]{};
    std::atomic<const Impl *> impl{nullptr};
    Impl generic, spec;
    std::atomic<int> state{ST_PENDING};
    std::mutex mu;
    std::condition_variable cv;
    CUlibrary lib = nullptr;
    CUdeviceptr wait_count = 0;   // the module's cj_wait_timeouts, if it has bounded waits
    std::string name_expr, name_expr2, error;
    std::string custom_src;   // plan dispatchers: the generated translation unit
    double compile_ms = 0;
};

struct cj_group_plan_s;

namespace {

struct State {
    bool inited = false;
    int device = -1;
    bool compile_only = false;
    cj_config cfg{};
    int num_sms = 0;
    int smem_optin = 0;
    std::mutex mu;  // cache, queue, plans
    std::unordered_map<std::string, cj_handle_s *> cache;
    std::deque<cj_handle_s *> queue;
    std::condition_variable qcv;
    bool stop = false;
    int busy = 0;
    std::condition_variable idle_cv;
    std::vector<std::thread> workers;
    CUfunction gen_chain[2]{}, gen_lt[2]{}, gen_grp[2]{}, gen_eig[2]{}, gen_mass[2]{};
    struct Aot {
        cjint::AotKernel k;
        CUfunction fn;
    };
    std::vector<Aot> aot;
    std::vector<cj_group_plan_s *> plans;
    // statistics
    std::atomic<uint64_t> requests{0}, hits{0}, ok{0}, failed{0}, aot_hits{0};
    std::atomic<uint64_t> l_gen{0}, l_aot{0}, l_jit{0}, l_tma{0}, l_tma_fb{0}, l_disp{0};
    std::mutex smu;
    std::vector<double> compile_ms;
    std::vector<double> lookup_ns;
    size_t lookup_pos = 0;
    // cost-model decisions per request (key with tile 0), so the model runs
    // once per distinct request and never on the lookup path of a hit
    std::unordered_map<std::string, std::array<int, 4>> decisions;
    // A process that exits without cj_shutdown still stops its compile
    // threads here (no CUDA calls: the runtime may already be gone).
    ~State() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
            queue.clear();
        }
        qcv.notify_all();
        for (auto &t : workers)
            if (t.joinable()) t.join();
    }
} G;

std::mutex g_init_mu;

int esize(int dtype) { return dtype == CJ_F64 ? 8 : 4; }
int dt_index(int dtype) { return dtype == CJ_F64 ? 0 : 1; }
const char *ctype(int dtype) { return dtype == CJ_F64 ? "double" : "float"; }

// ---------------------------------------------------------------------------
// Requests: validation, normalisation, default tiles, canonical key
// ---------------------------------------------------------------------------
bool g_fast(int lay) { return lay == 1 || lay == 4; }
bool z_fast(int lay) { return lay == 0 || lay == 2; }
// Axis (0 = d or m, 1 = g, 2 = z) at slot s (0 slowest .. 2 fastest) of storage order lay.
int lt_axis_host(int lay, int s) {
    static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    return order[lay][s];
}
bool is_lt(int k) { return k == CJ_K_LTIMES || k == CJ_K_LPLUSTIMES; }
// Shared-memory operand stages of the mode-4 twin that a TMA-fed tcgen05
// LTimes tile (mode 5 or 6) runs where `in` admits no tensor map: mode 5's
// own stage count; two for mode 6, whose stages are in tensor memory.
int lt_twin_stages(const cj_template_args &a) {
    return ((a.tile[3] >> 16) & 0xf) == 6 ? 2 : (a.tile[3] >> 8) & 0xff;
}
// Its producer warps: mode 5's converter count (at most 8: register producers
// split a stage's 8 direction quads over warps); 8 for mode 6.
int lt_twin_producers(const cj_template_args &a) {
    return ((a.tile[3] >> 16) & 0xf) == 6 ? 8 : std::min(a.tile[3] & 0xff, 8);
}
bool is_eig(int k) { return k == CJ_K_EIGEN_RECURRENCE; }
bool is_mass(int k) { return k == CJ_K_MASS; }
// Mass operator default: elements per block filling about 256 threads, both
// buffers of every element within 96 KiB.
int mass_default_epb(int dim, int D, int Q, int es) {
    const int m = cjg::mass_m(D, Q);
    int epb = std::max(1, 256 / (m * m));
    while (epb > 1 && cjg::mass_smem(dim, D, Q, epb, es) > 96 * 1024) --epb;
    return epb;
}
// Eigen recurrence default: f32 with n >= 2 two rows per thread (mapping 2),
// else one; instances per block up to 128 threads, both buffers within 96 KiB.
int eig_default_map(int n, int dtype) { return dtype == CJ_F32 && n >= 2 ? 2 : 1; }
int eig_default_ipb(int n, int es, int map = 1) {
    const int tpi = map == 2 ? (n + 1) / 2 : n;
    int ipb = std::max(1, 128 / tpi);
    while (ipb > 1 && cjg::eig_smem(n, ipb, es, map) > 96 * 1024) --ipb;
    return ipb;
}

// The LTimes kernel a request runs: LPlusTimes is LTimes of the swapped
// problem (output rows d, contracted m, orders exchanged) with accumulation.
struct LtView {
    int m, d, lin, lout, acc;
};
LtView lt_view(int k, const cj_template_args &a) {
    if (k == CJ_K_LPLUSTIMES) return {a.d, a.m, a.layout_b, a.layout_a, 1};
    return {a.m, a.d, a.layout_a, a.layout_b, 0};
}

void default_tile(int k, cj_template_args &a) {
    if (is_mass(k)) {
        // 2-D elements small enough for one thread each run that way (form 2,
        // 128 per block): 1.3-3.4x the shared-memory form in FP32 and up to
        // 1.7x in FP64 on the 2 GB cases
        if (cjg::mass_thread_ok(a.d, a.n, a.m)) {
            a.tile[0] = 128;
            a.tile[1] = 2;
        } else {
            a.tile[0] = mass_default_epb(a.d, a.n, a.m, esize(a.dtype));
            a.tile[1] = 0;
        }
        a.tile[2] = a.tile[3] = 0;
        return;
    }
    if (is_eig(k)) {
        a.tile[0] = eig_default_map(a.n, a.dtype);
        a.tile[1] = eig_default_ipb(a.n, esize(a.dtype), a.tile[0]);
        a.tile[2] = a.tile[3] = 0;
        return;
    }
    if (!is_lt(k)) {
        a.tile[0] = cjint::chain_default_map(a.n, a.dtype);
        a.tile[1] = cjint::chain_default_ipb(a.n, a.dtype);
        a.tile[2] = a.tile[3] = 0;
        if (k == CJ_K_UPDATE_CHAIN_GROUPED && a.dtype == CJ_F32 && a.n >= 17) {
            // uneven batches hold few large instances: one per block, on
            // (n / 4)^2 threads (register blocks), shortens the longest chain
            a.tile[0] = 5;
            a.tile[1] = 1;
        }
        return;
    }
    const int ct = 64;
    const LtView v = lt_view(k, a);
    const bool gi = g_fast(v.lin), go = g_fast(v.lout);
    int tg;
    if (!gi && !go) tg = 1;
    else if ((gi && z_fast(v.lout)) || (go && z_fast(v.lin))) tg = 8;
    else tg = 32;
    a.tile[0] = tg;
    a.tile[1] = ct / tg;
    if (a.dtype == CJ_F32 && v.m <= 128) {
        // tcgen05 3xTF32, 128 columns, fed by TMA with the deepest box ring
        // (6 .. 2) that fits in shared memory: operands in tensor memory (mode
        // 6: 4 TMEM stages, 4 converter warps), else in shared memory (mode 5:
        // 2 stages, 8 converter warps); else register producers (mode 4).
        // The box shape rule above keeps in's innermost box extent a multiple
        // of 4.
        a.tile[1] = 128 / tg;
        const int npa = (cjg::lt_tc_np(v.m) + 31) / 32 * 32;
        if (2 * npa + 64 * 4 <= 512 && cjg::lt_tc_smem(v.m, v.d, 2, tg, 128 / tg, v.lout) <= 220 * 1024)
            for (int boxes = 6; boxes >= 2; --boxes)
                if (cjg::lt_tc_smem(v.m, v.d, 0, tg, 128 / tg, v.lout, boxes) <= 220 * 1024) {
                    a.tile[2] = 32 * (6 + 4);
                    a.tile[3] = (boxes << 20) | (6 << 16) | (4 << 8) | 4;
                    return;
                }
        for (int boxes = 4; boxes >= 2; --boxes)
            if (cjg::lt_tc_smem(v.m, v.d, 2, tg, 128 / tg, v.lout, boxes) <= 220 * 1024) {
                a.tile[2] = 32 * (6 + 8);
                a.tile[3] = (boxes << 20) | (5 << 16) | (2 << 8) | 8;
                return;
            }
        if (cjg::lt_tc_smem(v.m, v.d, 2, tg, 128 / tg, v.lout) <= 220 * 1024) {
            a.tile[2] = 32 * (5 + 8);
            a.tile[3] = (4 << 16) | (2 << 8) | 8;
            return;
        }
    }
    if (a.dtype == CJ_F32) {
        // 64 columns, R 2, S 12, pipelined loads; threads = 32 * ceil(m / 12)
        a.tile[0] = tg;
        a.tile[1] = 64 / tg;
        a.tile[2] = 32 * ((v.m + 11) / 12);
        a.tile[3] = (1 << 20) | (2 << 8) | 12;
        return;
    }
    // other f64: R 1, S 9; threads = CT * ceil(m / 9)
    a.tile[2] = ct * ((v.m + 8) / 9);
    a.tile[3] = (1 << 8) | 9;
}

void put16(unsigned char *p, uint32_t v) { p[0] = v & 0xff; p[1] = (v >> 8) & 0xff; }
void put32(unsigned char *p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (v >> (8 * i)) & 0xff; }

void make_key(int k, const cj_template_args &a, unsigned char *key) {
    memset(key, 0, 32);
    put16(key + 0, (uint32_t)k);
    key[2] = (unsigned char)a.dtype;
    key[3] = (unsigned char)a.layout_a;
    key[4] = (unsigned char)a.layout_b;
    put16(key + 6, (uint32_t)a.n);
    put16(key + 8, (uint32_t)a.m);
    put16(key + 10, (uint32_t)a.d);
    for (int i = 0; i < 4; ++i) put32(key + 12 + 4 * i, (uint32_t)a.tile[i]);
    put32(key + 28, a.flags & kKeyFlags);
}

cj_status validate_and_normalise(int k, const cj_template_args &in, cj_template_args &a) {
    a = in;
    if (k != CJ_K_UPDATE_CHAIN && k != CJ_K_LTIMES && k != CJ_K_UPDATE_CHAIN_GROUPED && k != CJ_K_LPLUSTIMES &&
        k != CJ_K_EIGEN_RECURRENCE && k != CJ_K_MASS)
        return fail(CJ_ERR_INVALID_ARG, "unknown kernel id %d", k);
    if (a.dtype < 0 || a.dtype > 2) return fail(CJ_ERR_INVALID_ARG, "dtype %d out of range", a.dtype);
    if (a.flags & ~kKeyFlags) return fail(CJ_ERR_INVALID_ARG, "unknown flag bits 0x%x", a.flags & ~kKeyFlags);
    if (is_lt(k)) {
        if (a.dtype == CJ_BF16) return fail(CJ_ERR_INVALID_ARG, "LTimes supports f64 and f32 only");
        if (a.layout_a < 0 || a.layout_a > 5 || a.layout_b < 0 || a.layout_b > 5)
            return fail(CJ_ERR_INVALID_ARG, "LTimes storage orders must be 0..5");
        if (a.m < 1 || a.m > 64 || a.d < 1 || a.d > 128)
            return fail(CJ_ERR_INVALID_ARG, "LTimes needs 1 <= m <= 64 and 1 <= d <= 128");
        a.n = 0;
    } else if (is_mass(k)) {
        if (a.dtype == CJ_BF16) return fail(CJ_ERR_INVALID_ARG, "the mass operator supports f64 and f32 only");
        if (a.d != 2 && a.d != 3) return fail(CJ_ERR_INVALID_ARG, "mass operator dimension d = %d must be 2 or 3", a.d);
        if (a.n < 1 || a.n > 16 || a.m < 1 || a.m > 16)
            return fail(CJ_ERR_INVALID_ARG, "mass operator needs 1 <= n (dofs per dimension) <= 16 and "
                                            "1 <= m (quadrature points per dimension) <= 16");
        a.layout_a = a.layout_b = 0;
    } else if (is_eig(k)) {
        if (a.n < 1 || a.n > 32) return fail(CJ_ERR_INVALID_ARG, "Eigen recurrence n = %d outside 1..32", a.n);
        if (a.dtype == CJ_BF16) return fail(CJ_ERR_INVALID_ARG, "the Eigen recurrence supports f64 and f32 only");
        a.layout_a = a.layout_b = a.m = a.d = 0;   // row-major only
    } else {
        if (a.n < 1 || a.n > 64) return fail(CJ_ERR_INVALID_ARG, "n = %d outside 1..64", a.n);
        if (k == CJ_K_UPDATE_CHAIN_GROUPED) a.layout_a = 0;
        if (a.layout_a != 0 && a.layout_a != 1) return fail(CJ_ERR_INVALID_ARG, "layout %d must be 0 or 1", a.layout_a);
        if (a.dtype == CJ_BF16 && a.n < 16) return fail(CJ_ERR_INVALID_ARG, "bf16 needs n >= 16");
        a.m = a.d = a.layout_b = 0;
    }
    if ((a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT) && (!is_lt(k) || (a.flags & CJ_FLAG_GENERIC)))
        return fail(CJ_ERR_INVALID_ARG, "the wait-timeout hook applies to specialized LTimes kernels only");
    if (a.flags & CJ_FLAG_GENERIC) {
        for (int &t : a.tile) t = 0;
        return CJ_OK;
    }
    if (a.tile[0] == 0 && a.tile[1] == 0 && a.tile[2] == 0 && a.tile[3] == 0) {
        bool chosen = false;
        if (G.cfg.use_cost_model && !G.compile_only && (k == CJ_K_UPDATE_CHAIN || k == CJ_K_LTIMES)) {
            unsigned char rk[32];
            make_key(k, a, rk);
            const std::string rs(reinterpret_cast<char *>(rk), 32);
            {
                std::lock_guard<std::mutex> lk(G.mu);
                auto it = G.decisions.find(rs);
                if (it != G.decisions.end()) {
                    std::memcpy(a.tile, it->second.data(), sizeof a.tile);
                    chosen = true;
                }
            }
            if (!chosen && cjint::cost_model_tile(k, a, a.tile)) {
                chosen = true;
                std::array<int, 4> t{a.tile[0], a.tile[1], a.tile[2], a.tile[3]};
                std::lock_guard<std::mutex> lk(G.mu);
                G.decisions.emplace(rs, t);
            }
        }
        if (!chosen) default_tile(k, a);
    }
    // explicit tiles: check the kernel can be instantiated and launched
    if (is_mass(k)) {
        if (a.tile[0] < 1 || a.tile[1] < 0 || a.tile[1] > 2 || a.tile[2] || a.tile[3] ||
            (a.tile[1] == 2 && !cjg::mass_thread_ok(a.d, a.n, a.m)) ||
            cjg::mass_threads(a.n, a.m, a.tile[0], a.tile[1]) > 1024 ||
            cjg::mass_smem(a.d, a.n, a.m, a.tile[0], esize(a.dtype), a.tile[1]) > 220 * 1024)
            return fail(CJ_ERR_INVALID_ARG, "mass operator tile {%d,%d,%d,%d} invalid ({elements per block, form: 0 "
                        "one group per block, 1 persistent with staged loads, 2 one thread per element (2-D, "
                        "D Q + D^2 <= 80), 0, 0}, at most 1024 threads and 220 KiB of shared memory)",
                        a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        return CJ_OK;
    }
    if (is_eig(k)) {
        // mapping 1: one row per thread; 2: two rows per thread (f32)
        const int map = a.tile[0];
        if ((map != 1 && !(map == 2 && a.dtype == CJ_F32)) || a.tile[1] < 1 || a.tile[2] || a.tile[3] ||
            cjg::chain_threads(a.n, map == 2 ? 6 : 1, a.tile[1]) > 1024 ||
            cjg::eig_smem(a.n, a.tile[1], esize(a.dtype), map) > 220 * 1024)
            return fail(CJ_ERR_INVALID_ARG,
                        "Eigen recurrence tile {%d,%d,%d,%d} invalid ({1, or 2 for f32; instances per block, 0, 0})",
                        a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        return CJ_OK;
    }
    if (!is_lt(k)) {
        const int map = a.tile[0], ipb = a.tile[1];
        if (map < 1 || map > 8) return fail(CJ_ERR_INVALID_ARG, "update chain mapping %d must be 1..8", map);
        if (map == 6 && a.dtype != CJ_F32)
            return fail(CJ_ERR_INVALID_ARG, "mapping 6 (two rows per thread) needs f32");
        if ((map == 5 || map == 8) && (a.dtype != CJ_F32 || a.n < 8))
            return fail(CJ_ERR_INVALID_ARG, "mappings 5 and 8 (register blocks) need f32 and n >= 8");
        if ((map == 3 || map == 7) != (a.dtype == CJ_BF16))
            return fail(CJ_ERR_INVALID_ARG, "mappings 3 and 7 (bf16 tensor cores) are the mappings of dtype bf16");
        if (map == 7 && (ipb != 1 || (a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT)))
            return fail(CJ_ERR_INVALID_ARG, "mapping 7 (tcgen05) takes one instance per block");
        if (map == 2 && a.n > 8) return fail(CJ_ERR_INVALID_ARG, "mapping 2 needs n <= 8");
        if (map == 4 && !cjint::chain_dmma_ok(a.n, a.dtype))
            return fail(CJ_ERR_INVALID_ARG, "mapping 4 (FP64 tensor cores) needs f64 and n in {8, 16, 24, 32}");
        if (ipb < 1 || cjg::chain_threads(a.n, map, ipb) > 1024 || a.tile[2] || a.tile[3])
            return fail(CJ_ERR_INVALID_ARG, "bad instances-per-block %d for n = %d", ipb, a.n);
        if (k == CJ_K_UPDATE_CHAIN_GROUPED && ipb > 256) return fail(CJ_ERR_INVALID_ARG, "grouped ipb must be <= 256");
        if (cjg::chain_smem(a.n, map, ipb, esize(a.dtype)) > 220 * 1024)
            return fail(CJ_ERR_INVALID_ARG, "tile needs too much shared memory");
    } else {
        const int tg = a.tile[0], tz = a.tile[1], nt = a.tile[2];
        const LtView v = lt_view(k, a);
        const int pipe = (a.tile[3] >> 20) & 0xf, mode = (a.tile[3] >> 16) & 0xf;
        const int r = (a.tile[3] >> 8) & 0xff, s = a.tile[3] & 0xff;
        // modes 4-6 reuse the pipe field: producers' prefetch depth (0 = automatic) / TMA ring depth
        if ((mode >= 4 && mode <= 6 ? pipe > 8 : pipe > 1) || (a.tile[3] >> 24))
            return fail(CJ_ERR_INVALID_ARG, "LTimes tile flags 0x%x unknown", a.tile[3]);
        if (mode == 1 && (a.dtype != CJ_F64 || s != 8 || v.d % 4 || r < 1 || (tg * tz) % (8 * r) ||
                          (tg * tz / (8 * r)) * 32 != nt || nt > 1024))
            return fail(CJ_ERR_INVALID_ARG, "LTimes tensor-core tile {%d,%d,%d,0x%x} invalid (f64, S = 8, d %% 4 == 0, "
                        "threads = 32 * TG * TZ / (8 R))", a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        if (mode == 2 && (a.dtype != CJ_F32 || s != 8 || r != 1 || v.d % 8 || (tg * tz) % 16 ||
                          (tg * tz / 16) * 32 != nt || nt > 1024))
            return fail(CJ_ERR_INVALID_ARG, "LTimes 3xTF32 tile {%d,%d,%d,0x%x} invalid (f32, R = 1, S = 8, d %% 8 == 0, "
                        "threads = 32 * TG * TZ / 16)", a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        const int direct_groups = s ? (v.m + s - 1) / s : 1;   // moment groups of the direct kernel
        if (mode == 3 && (a.dtype != CJ_F32 || pipe || r < 1 || r > 4 || (s != 0 && (s % 4 || s >= v.m)) ||
                          (tg * tz) % r || (tg * tz / r) * direct_groups != nt || nt < 32 || nt > 1024))
            return fail(CJ_ERR_INVALID_ARG, "LTimes direct tile {%d,%d,%d,0x%x} invalid (f32, no PIPE, R <= 4, S = 0 "
                        "or a multiple of 4 below m, threads = TG * TZ / R * ceil(m / S))", a.tile[0], a.tile[1],
                        a.tile[2], a.tile[3]);
        if (mode == 4 && (a.dtype != CJ_F32 || tg * tz != 128 || r < 2 || r > 8 ||
                          (s != 2 && s != 4 && s != 8) || nt != 32 * (5 + s) || v.m > 128))
            return fail(CJ_ERR_INVALID_ARG, "LTimes tcgen05 tile {%d,%d,%d,0x%x} invalid (f32, TG * TZ = 128, "
                        "2 <= stages <= 8, producer warps 2/4/8, threads = 32 * (5 + producer warps), m <= 128)",
                        a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        if (mode == 5) {
            const int inner = lt_axis_host(v.lin, 2);   // innermost axis of `in`: its TMA box extent
            const int ib = inner == 0 ? 32 : inner == 1 ? tg : tz;
            if (a.dtype != CJ_F32 || tg * tz != 128 || r < 2 || r > 8 || (s != 2 && s != 4 && s != 8) ||
                nt != 32 * (6 + s) || v.m > 128 || pipe < 2 || ib % 4)
                return fail(CJ_ERR_INVALID_ARG, "LTimes tcgen05+TMA tile {%d,%d,%d,0x%x} invalid (f32, TG * TZ = 128, "
                            "2 <= stages <= 8, converter warps 2/4/8, threads = 32 * (6 + converter warps), "
                            "2 <= TMA boxes <= 8, in's innermost box extent a multiple of 4, m <= 128)",
                            a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        }
        if (mode == 6) {
            // TMEM operand stages of 64 columns after two accumulators, at most 512 columns in all
            const int inner = lt_axis_host(v.lin, 2);
            const int ib = inner == 0 ? 32 : inner == 1 ? tg : tz;
            const int npa = (cjg::lt_tc_np(v.m) + 31) / 32 * 32;
            if (a.dtype != CJ_F32 || tg * tz != 128 || r < 2 || 2 * npa + 64 * r > 512 || (s != 4 && s != 8) ||
                nt != 32 * (6 + s) || v.m > 128 || pipe < 2 || ib % 4 ||
                cjg::lt_tc_smem(v.m, v.d, 2, tg, tz, v.lout) > 220 * 1024)   // and its mode-4 twin fits
                return fail(CJ_ERR_INVALID_ARG, "LTimes tcgen05 TMEM-operand tile {%d,%d,%d,0x%x} invalid (f32, TG * "
                            "TZ = 128, converter warps 4/8, threads = 32 * (6 + converter warps), 2 <= TMA boxes "
                            "<= 8, in's innermost box extent a multiple of 4, m <= 128, 2 <= stages and "
                            "2 * ceil32(ceil16(m)) + 64 * stages <= 512 TMEM columns)",
                            a.tile[0], a.tile[1], a.tile[2], a.tile[3]);
        }
        if (mode > 6) return fail(CJ_ERR_INVALID_ARG, "LTimes compute mode %d unknown", mode);
        if ((a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT) && mode < 4)
            return fail(CJ_ERR_INVALID_ARG, "the wait-timeout hook applies to tile modes 4-6 only");
        if (mode == 0 && (tg < 1 || tz < 1 || r < 1 || s < 1 || nt < 32 || nt > 1024 || (tg * tz) % r ||
                          (tg * tz / r) * ((v.m + s - 1) / s) != nt))
            return fail(CJ_ERR_INVALID_ARG, "LTimes tile {%d,%d,%d,%d} does not cover its block", a.tile[0],
                        a.tile[1], a.tile[2], a.tile[3]);
        if ((mode == 6   ? cjg::lt_tc_smem(v.m, v.d, 0, tg, tz, v.lout, pipe)
             : mode == 5 ? cjg::lt_tc_smem(v.m, v.d, r, tg, tz, v.lout, pipe)
             : mode == 4 ? cjg::lt_tc_smem(v.m, v.d, r, tg, tz, v.lout)
             : mode == 3 ? cjg::lt_direct_smem(v.m, v.d, tg * tz, esize(a.dtype), s)
                         : cjg::lt_smem(v.m, s, v.d, tg * tz, esize(a.dtype), pipe, mode)) > 220 * 1024)
            return fail(CJ_ERR_INVALID_ARG, "LTimes tile needs too much shared memory");
    }
    return CJ_OK;
}

// ---------------------------------------------------------------------------
// Launch geometry
// ---------------------------------------------------------------------------
int occupancy(CUfunction f, int threads, size_t smem) {
    int nb = 1;
    if (f && drv.OccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != CUDA_SUCCESS) nb = 1;
    return nb < 1 ? 1 : nb;
}

void generic_impl(cj_handle_s *h) {
    Impl &g = h->generic;
    const cj_template_args &a = h->a;
    const int di = dt_index(a.dtype), es = esize(a.dtype);
    g.variant = V_GENERIC;
    if (is_mass(h->kernel)) {
        g.fn = G.gen_mass[di];
        g.ipb = mass_default_epb(a.d, a.n, a.m, es);
        g.threads = cjg::mass_threads(a.n, a.m, g.ipb);
        g.smem = (size_t)cjg::mass_smem(a.d, a.n, a.m, g.ipb, es);
    } else if (is_eig(h->kernel)) {
        g.fn = G.gen_eig[di];
        g.ipb = eig_default_ipb(a.n, es);
        g.threads = cjg::chain_threads(a.n, 1, g.ipb);
        g.smem = (size_t)cjg::eig_smem(a.n, g.ipb, es);
    } else if (is_lt(h->kernel)) {
        const LtView v = lt_view(h->kernel, a);
        g.fn = G.gen_lt[di];
        g.threads = a.dtype == CJ_F64 ? 64 : 128;
        g.smem = (size_t)cjg::lt_generic_smem(v.m, v.d, g.threads, es);
    } else {
        g.fn = h->kernel == CJ_K_UPDATE_CHAIN ? G.gen_chain[di] : G.gen_grp[di];
        g.ipb = std::max(1, 128 / a.n);
        g.threads = ((g.ipb * a.n + 31) / 32) * 32;
        g.smem = (size_t)cjg::chain_generic_smem(a.n, g.ipb, g.threads, es);
        if (h->kernel == CJ_K_UPDATE_CHAIN_GROUPED) g.blocks_per_sm = occupancy(g.fn, g.threads, g.smem);
    }
}

// Internal kernel id of a plan dispatcher (never a request; no 32-byte key).
constexpr int kDispatchKernel = 100;

void spec_geometry(const cj_handle_s *h, Impl &s) {
    const cj_template_args &a = h->a;
    const int es = esize(a.dtype);
    if (h->kernel == kDispatchKernel) {
        s.threads = a.tile[0];
        s.smem = (size_t)a.tile[1];
    } else if (is_mass(h->kernel)) {
        s.ipb = a.tile[0];
        s.threads = cjg::mass_threads(a.n, a.m, a.tile[0], a.tile[1]);
        s.smem = (size_t)cjg::mass_smem(a.d, a.n, a.m, a.tile[0], es, a.tile[1]);
    } else if (is_eig(h->kernel)) {
        s.ipb = a.tile[1];
        s.threads = cjg::chain_threads(a.n, a.tile[0] == 2 ? 6 : 1, a.tile[1]);
        s.smem = (size_t)cjg::eig_smem(a.n, a.tile[1], es, a.tile[0]);
    } else if (is_lt(h->kernel)) {
        const LtView v = lt_view(h->kernel, a);
        const int mode = (a.tile[3] >> 16) & 0xf;
        s.threads = a.tile[2];
        if (mode == 5 || mode == 6) {   // and its mode-4 twin
            s.threads2 = 32 * (5 + lt_twin_producers(a));
            s.smem2 = (size_t)cjg::lt_tc_smem(v.m, v.d, lt_twin_stages(a), a.tile[0], a.tile[1], v.lout);
        }
        s.smem = mode == 6   ? (size_t)cjg::lt_tc_smem(v.m, v.d, 0, a.tile[0], a.tile[1], v.lout, (a.tile[3] >> 20) & 0xf)
                 : mode == 5 ? (size_t)cjg::lt_tc_smem(v.m, v.d, (a.tile[3] >> 8) & 0xff, a.tile[0], a.tile[1], v.lout,
                                                       (a.tile[3] >> 20) & 0xf)
                 : mode == 4 ? (size_t)cjg::lt_tc_smem(v.m, v.d, (a.tile[3] >> 8) & 0xff, a.tile[0], a.tile[1], v.lout)
                 : mode == 3 ? (size_t)cjg::lt_direct_smem(v.m, v.d, a.tile[0] * a.tile[1], es, a.tile[3] & 0xff)
                             : (size_t)cjg::lt_smem(v.m, a.tile[3] & 0xff, v.d, a.tile[0] * a.tile[1], es,
                                                    (a.tile[3] >> 20) & 1, mode);
    } else {
        s.ipb = a.tile[1];
        s.threads = cjg::chain_threads(a.n, a.tile[0], a.tile[1]);
        s.smem = (size_t)cjg::chain_smem(a.n, a.tile[0], a.tile[1], es);
    }
}

// Modes 5 and 6 also compile their mode-4 twin (register producers) into the
// module.
std::string fallback_name_expression(const cj_handle_s *h) {
    const cj_template_args &a = h->a;
    const int mode = (a.tile[3] >> 16) & 0xf;
    if (!is_lt(h->kernel) || (mode != 5 && mode != 6)) return "";
    const LtView v = lt_view(h->kernel, a);
    char buf[256];
    snprintf(buf, sizeof buf, "cj::ltimes_tc<%d, %d, %d, %d, %d, %d, %d, %d, 0, 0, %d, %d>", v.m, v.d, v.lin, v.lout,
             a.tile[0], a.tile[1], lt_twin_stages(a), lt_twin_producers(a), v.acc,
             (a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT) ? 1 : 0);
    return buf;
}

std::string name_expression(const cj_handle_s *h) {
    const cj_template_args &a = h->a;
    char buf[256];
    if (h->kernel == CJ_K_UPDATE_CHAIN && a.tile[0] == 7)
        snprintf(buf, sizeof buf, "cj::update_chain_tc<%d, %d>", a.n, a.layout_a);
    else if (h->kernel == CJ_K_UPDATE_CHAIN_GROUPED && a.tile[0] == 7)
        snprintf(buf, sizeof buf, "cj::update_chain_grouped_tc<%d>", a.n);
    else if (h->kernel == CJ_K_UPDATE_CHAIN)
        snprintf(buf, sizeof buf, "cj::update_chain<%s, %d, %d, %d, %d>", ctype(a.dtype), a.n, a.layout_a,
                 a.tile[0], a.tile[1]);
    else if (is_mass(h->kernel))
        if (a.tile[1] == 2)
            snprintf(buf, sizeof buf, "cj::mass_apply_thread<%s, %d, %d, %d>", ctype(a.dtype), a.n, a.m, a.tile[0]);
        else
            snprintf(buf, sizeof buf, "cj::mass_apply%s<%s, %d, %d, %d, %d>", a.tile[1] ? "_pipe" : "",
                     ctype(a.dtype), a.d, a.n, a.m, a.tile[0]);
    else if (is_eig(h->kernel))
        snprintf(buf, sizeof buf, "cj::eigen_recurrence%s<%s, %d, %d>", a.tile[0] == 2 ? "2" : "", ctype(a.dtype),
                 a.n, a.tile[1]);
    else if (h->kernel == CJ_K_UPDATE_CHAIN_GROUPED)
        snprintf(buf, sizeof buf, "cj::update_chain_grouped<%s, %d, %d, %d>", ctype(a.dtype), a.n, a.tile[0],
                 a.tile[1]);
    else {
        const LtView v = lt_view(h->kernel, a);
        const int mode = (a.tile[3] >> 16) & 0xf;
        if (mode == 4 || mode == 5)   // mode 5: the pipe field is the TMA ring depth; mode 4: the prefetch depth
            snprintf(buf, sizeof buf, "cj::ltimes_tc<%d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d>", v.m, v.d,
                     v.lin, v.lout, a.tile[0], a.tile[1], (a.tile[3] >> 8) & 0xff, a.tile[3] & 0xff,
                     mode == 4 ? (a.tile[3] >> 20) & 0xf : 0, mode == 5 ? (a.tile[3] >> 20) & 0xf : 0, v.acc,
                     (a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT) ? 1 : 0);
        else if (mode == 6)   // TMA ring depth in the pipe field, operand stages in TMEM
            snprintf(buf, sizeof buf, "cj::ltimes_tc<%d, %d, %d, %d, %d, %d, %d, %d, 0, %d, %d, %d, 1>", v.m, v.d,
                     v.lin, v.lout, a.tile[0], a.tile[1], (a.tile[3] >> 8) & 0xff, a.tile[3] & 0xff,
                     (a.tile[3] >> 20) & 0xf, v.acc, (a.flags & CJ_FLAG_INJECT_WAIT_TIMEOUT) ? 1 : 0);
        else if (((a.tile[3] >> 16) & 0xf) == 3)
            snprintf(buf, sizeof buf, "cj::ltimes_direct<%s, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d>", ctype(a.dtype),
                     v.m, v.d, v.lin, v.lout, a.tile[0], a.tile[1], a.tile[2], (a.tile[3] >> 8) & 0xff,
                     a.tile[3] & 0xff, v.acc);
        else
            snprintf(buf, sizeof buf, "cj::ltimes<%s, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d>", ctype(a.dtype),
                     v.m, v.d, v.lin, v.lout, a.tile[0], a.tile[1], a.tile[2], (a.tile[3] >> 8) & 0xff,
                     a.tile[3] & 0xff, (a.tile[3] >> 16) & 0xf, (a.tile[3] >> 20) & 0xf, v.acc);
    }
    return buf;
}

// ---------------------------------------------------------------------------
// NVRTC specializer: in-memory sources and headers only.
// ---------------------------------------------------------------------------
// --no-cache: NVRTC would otherwise read and write the per-user CUDA compute
// cache (~/.nv/ComputeCache) when a driver is present; the paper's design
// requirement is that run-time compilation touches no file (Sec. 1).
const char *kNvrtcOpts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "--no-cache"};
constexpr int kNumNvrtcOpts = 4;

struct CompileOut {
    nvrtcResult rc = NVRTC_SUCCESS;
    std::string log, lowered, lowered2;
    std::vector<char> cubin;
};

CompileOut nvrtc_compile(const std::string &src, const char *name_expr, const char *name_expr2 = nullptr) {
    CompileOut out;
    const char *hdr_src[5] = {cj_emb_geometry_h, cj_emb_update_chain_cuh, cj_emb_ltimes_cuh, cj_emb_mass_cuh,
                              cj_emb_chain_tc_cuh};
    const char *hdr_name[5] = {"geometry.h", "update_chain.cuh", "ltimes.cuh", "mass.cuh", "chain_tc.cuh"};
    nvrtcProgram prog;
    out.rc = nvrtcCreateProgram(&prog, src.c_str(), "cj_instantiation.cu", 5, hdr_src, hdr_name);
    if (out.rc != NVRTC_SUCCESS) return out;
    if (name_expr) nvrtcAddNameExpression(prog, name_expr);
    if (name_expr2) nvrtcAddNameExpression(prog, name_expr2);
    out.rc = nvrtcCompileProgram(prog, kNumNvrtcOpts, kNvrtcOpts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    if (ls > 1) {
        out.log.resize(ls);
        nvrtcGetProgramLog(prog, &out.log[0]);
    }
    if (out.rc == NVRTC_SUCCESS) {
        if (name_expr) {
            const char *low = nullptr;
            out.rc = nvrtcGetLoweredName(prog, name_expr, &low);
            if (out.rc == NVRTC_SUCCESS && low) out.lowered = low;
        }
        if (out.rc == NVRTC_SUCCESS && name_expr2) {
            const char *low = nullptr;
            out.rc = nvrtcGetLoweredName(prog, name_expr2, &low);
            if (out.rc == NVRTC_SUCCESS && low) out.lowered2 = low;
        }
        size_t cs = 0;
        if (out.rc == NVRTC_SUCCESS) out.rc = nvrtcGetCUBINSize(prog, &cs);
        if (out.rc == NVRTC_SUCCESS) {
            out.cubin.resize(cs);
            out.rc = nvrtcGetCUBIN(prog, out.cubin.data());
        }
    }
    nvrtcDestroyProgram(&prog);
    return out;
}

void record_compile_ms(double ms) {
    std::lock_guard<std::mutex> lk(G.smu);
    G.compile_ms.push_back(ms);
}

void finish(cj_handle_s *h, int state) {
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->state.store(state, std::memory_order_release);
    }
    h->cv.notify_all();
}

cj_status compile_handle(cj_handle_s *h) {
    const auto t0 = clk::now();
    std::string src = !h->custom_src.empty() ? h->custom_src
                      : is_lt(h->kernel)      ? "#include \"ltimes.cuh\"\n"
                      : is_mass(h->kernel)    ? "#include \"mass.cuh\"\n"
                      : h->a.tile[0] == 7     ? "#include \"chain_tc.cuh\"\n"
                                              : "#include \"update_chain.cuh\"\n";
    if (h->a.flags & CJ_FLAG_INJECT_COMPILE_ERROR)
        src += "namespace cj { __device__ int injected_failure = this_identifier_does_not_exist; }\n";
    CompileOut c = nvrtc_compile(src, h->name_expr.c_str(), h->name_expr2.empty() ? nullptr : h->name_expr2.c_str());
    if (c.rc != NVRTC_SUCCESS) {
        h->error = std::string("NVRTC: ") + nvrtcGetErrorString(c.rc) + "\n" + c.log;
        t_err = h->error;
        G.failed++;
        finish(h, ST_FAILED);
        return CJ_ERR_COMPILE;
    }
    Impl &s = h->spec;
    spec_geometry(h, s);
    s.variant = V_JIT;
    if (!G.compile_only) {
        cudaSetDevice(G.device);
        CUkernel kern = nullptr;
        CUresult r = drv.LibraryLoadData(&h->lib, c.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (r == CUDA_SUCCESS) r = drv.LibraryGetKernel(&kern, h->lib, c.lowered.c_str());
        if (r == CUDA_SUCCESS) r = drv.KernelGetFunction(&s.fn, kern);
        if (r == CUDA_SUCCESS && s.smem > 48 * 1024)
            r = drv.FuncSetAttribute(s.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)s.smem);
        // a plan dispatcher's residency is set by its registers: let shared
        // memory take the whole carveout so that it never limits it further
        if (r == CUDA_SUCCESS && h->kernel == kDispatchKernel)
            r = drv.FuncSetAttribute(s.fn, CU_FUNC_ATTRIBUTE_PREFERRED_SHARED_MEMORY_CARVEOUT, 100);
        if (r == CUDA_SUCCESS && !c.lowered2.empty()) {
            CUkernel k2 = nullptr;
            r = drv.LibraryGetKernel(&k2, h->lib, c.lowered2.c_str());
            if (r == CUDA_SUCCESS) r = drv.KernelGetFunction(&s.fn2, k2);
            if (r == CUDA_SUCCESS && s.smem2 > 48 * 1024)
                r = drv.FuncSetAttribute(s.fn2, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)s.smem2);
            if (r == CUDA_SUCCESS) s.blocks2 = occupancy(s.fn2, s.threads2, s.smem2);
        }
        if (r != CUDA_SUCCESS) {
            h->error = std::string("module load: ") + cu_str(r);
            t_err = h->error;
            G.failed++;
            finish(h, ST_FAILED);
            return CJ_ERR_COMPILE;
        }
        s.blocks_per_sm = occupancy(s.fn, s.threads, s.smem);
        if (!is_lt(h->kernel) && !is_eig(h->kernel) && !is_mass(h->kernel) && h->kernel != kDispatchKernel &&
            h->a.tile[0] == 7) {
            // The occupancy query answers one block per SM for this kernel;
            // count the resident blocks from its registers, shared memory and
            // threads, capped so that their accumulator columns, held for the
            // block's life, fit the SM's 512 (an overcount only makes the
            // extra blocks wait for an SM)
            int regs = 0, stat = 0;
            drv.FuncGetAttribute(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, s.fn);
            drv.FuncGetAttribute(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, s.fn);
            const int warps = (s.threads + 31) / 32;
            const int by_regs = 65536 / std::max(1, warps * ((std::max(regs, 1) * 32 + 255) / 256 * 256));
            const int by_smem = (G.smem_optin + 1024) / (int)(s.smem + stat + 1024);
            s.blocks_per_sm = std::max(1, std::min({by_regs, by_smem, 64 / warps, 512 / (h->a.n <= 32 ? 32 : 64)}));
        }
        CUdeviceptr wp = 0;
        size_t wbytes = 0;
        if (drv.LibraryGetGlobal(&wp, &wbytes, h->lib, "cj_wait_timeouts") == CUDA_SUCCESS && wbytes == sizeof(uint32_t))
            h->wait_count = wp;
        h->impl.store(&h->spec, std::memory_order_release);
    }
    h->compile_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    record_compile_ms(h->compile_ms);
    G.ok++;
    finish(h, ST_READY);
    return CJ_OK;
}

// At process exit without cj_shutdown: stop the compile threads (a compile
// in flight finishes first).  Registered with atexit by cj_init, after the
// statically linked NVRTC and runtime have built their own static state, so
// it runs before their destructors; a thread still inside NVRTC while they
// ran would crash the process on its way out.
void stop_workers_at_exit() {
    {
        std::lock_guard<std::mutex> lk(G.mu);
        G.stop = true;
        G.queue.clear();
    }
    G.qcv.notify_all();
    for (auto &t : G.workers)
        if (t.joinable()) t.join();
    G.workers.clear();
}

void worker_loop() {
    if (!G.compile_only) cudaSetDevice(G.device);
    for (;;) {
        cj_handle_s *h;
        {
            std::unique_lock<std::mutex> lk(G.mu);
            G.qcv.wait(lk, [] { return G.stop || !G.queue.empty(); });
            if (G.stop || G.queue.empty()) return;   // shutdown drops compiles not yet started
            h = G.queue.front();
            G.queue.pop_front();
            G.busy++;
        }
        compile_handle(h);
        {
            std::lock_guard<std::mutex> lk(G.mu);
            G.busy--;
        }
        G.idle_cv.notify_all();
    }
}

// The explicit specialization for h's arguments, if one was compiled AoT.
const State::Aot *find_aot(const cj_handle_s *h) {
    for (const auto &e : G.aot)
        if (e.k.kernel == h->kernel && e.k.dtype == h->a.dtype && e.k.n == h->a.n && e.k.layout == h->a.layout_a &&
            e.k.tile[0] == h->a.tile[0] && e.k.tile[1] == h->a.tile[1])
            return &e;
    return nullptr;
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace

// ---------------------------------------------------------------------------
// Grouped plan
// ---------------------------------------------------------------------------
struct cj_group_plan_s {
    int dtype = 0;
    int64_t count = 0, pool_elems = 0;
    struct Group {
        int n = 0;
        cj_handle h = nullptr;
        int64_t n_items = 0, first_item = 0;
        double cost = 0;
    };
    std::vector<Group> groups;
    long long *d_items = nullptr;
    int *d_counters = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t capture = nullptr;   // graphs are captured here, then launched on the caller's stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_A = nullptr;
    void *g_X = nullptr;
    std::vector<const void *> g_impls;
    // the plan's dispatcher: one persistent kernel over every group, taking
    // cost-ordered tickets (chunks of one group) from counter ngroups
    cj_handle disp = nullptr;
    long long *d_tickets = nullptr;
    int n_tickets = 0;
    bool use_dispatcher = true;   // false once the plan's autotuner found the per-group form faster
    // every dispatcher variant requested for this plan, with its own tickets
    // (disp, d_tickets, n_tickets above are the one in use)
    struct DispForm {
        cj_handle h = nullptr;
        long long *d_tickets = nullptr;
        int n_tickets = 0;
    };
    std::vector<DispForm> disp_forms;
    std::vector<long long> h_items;   // the work list on the host
};

namespace {

void plan_free(cj_group_plan_s *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto s : p->streams) cudaStreamDestroy(s);
    for (auto e : p->join) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->capture) cudaStreamDestroy(p->capture);
    if (p->d_items) cudaFree(p->d_items);
    if (p->d_counters) cudaFree(p->d_counters);
    for (auto &f : p->disp_forms)
        if (f.d_tickets) cudaFree(f.d_tickets);
    delete p;
}

// The dispatcher's tile for a group of size n and dtype (the group's own:
// f32 for the n < 16 groups of a bf16 plan), for blocks of `block` threads:
// bf16 tensor-core panels (mapping 3); f32 n >= 8 register blocks (mapping
// 5); n <= 4 one instance per thread (mapping 2); otherwise one row per
// thread (mapping 1).  Rule 1 differs for f32 n >= 16: 4 x 8 register
// blocks (mapping 8).  As many instances per chunk as fill the block (at
// most 256), fewer where shared memory would exceed `smem_cap` bytes.
std::array<int, 2> dispatch_tile(int dtype, int n, int block, int rule, long smem_cap) {
    const int es = esize(dtype);
    int map, tpi;
    if (dtype == CJ_BF16) map = 3, tpi = ((n + 15) / 16) * 32;
    else if (dtype == CJ_F32 && n >= 16 && rule == 1) map = 8, tpi = ((n + 3) / 4) * ((n + 7) / 8);
    else if (dtype == CJ_F32 && n >= 8) map = 5, tpi = ((n + 3) / 4) * ((n + 3) / 4);
    else if (n <= 4) map = 2, tpi = 1;
    else map = 1, tpi = n;
    int ipb = std::max(1, std::min(256, block / tpi));
    while (ipb > 1 && (cjg::chain_threads(n, map, ipb) > block || cjg::chain_smem(n, map, ipb, es) > smem_cap))
        --ipb;
    return {map, ipb};
}

bool dispatcher_ready(const cj_group_plan_s *p) {
    return p->disp && p->disp->state.load(std::memory_order_acquire) == ST_READY &&
           p->disp->impl.load(std::memory_order_acquire) == &p->disp->spec;
}

cj_status plan_record(cj_group_plan_s *p, const void *A, void *X, cudaStream_t st, bool per_group) {
    if (cudaMemsetAsync(p->d_counters, 0, sizeof(int) * (p->groups.size() + 1), st) != cudaSuccess)
        return fail(CJ_ERR_CUDA, "grouped plan: counter reset failed");
    if (!per_group && p->use_dispatcher && dispatcher_ready(p)) {
        // one persistent launch for the whole batch
        const Impl *im = p->disp->impl.load(std::memory_order_acquire);
        const unsigned grid = (unsigned)std::min<long long>(p->n_tickets, (long long)G.num_sms * im->blocks_per_sm);
        void *tickets = p->d_tickets, *items = p->d_items, *counter = p->d_counters + p->groups.size();
        int nt = p->n_tickets;
        const void *a = A;
        void *x = X;
        void *args[6] = {&tickets, &nt, &items, &a, &x, &counter};
        const CUresult r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem,
                                            reinterpret_cast<CUstream>(st), args, nullptr);
        if (r != CUDA_SUCCESS) return fail(CJ_ERR_CUDA, "plan dispatcher launch failed: %s", cu_str(r));
        G.l_disp++;
        return CJ_OK;
    }
    if (cudaEventRecord(p->fork, st) != cudaSuccess)
        return fail(CJ_ERR_CUDA, "grouped plan: event record failed");
    for (size_t g = 0; g < p->groups.size(); ++g) {
        cudaStream_t s = p->streams[g % p->streams.size()];
        if (g < p->streams.size() && cudaStreamWaitEvent(s, p->fork, 0) != cudaSuccess)
            return fail(CJ_ERR_CUDA, "grouped plan: stream wait failed");
        const auto &gr = p->groups[g];
        void *items = p->d_items + 3 * gr.first_item;
        void *counter = p->d_counters + g;
        const void *a = A;
        void *x = X;
        void *args[4] = {&items, &a, &x, &counter};
        cj_status rc = cj_launch(gr.h, args, gr.n_items, s);
        if (rc != CJ_OK) return rc;
    }
    for (size_t i = 0; i < p->streams.size() && i < p->groups.size(); ++i) {
        if (cudaEventRecord(p->join[i], p->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(st, p->join[i], 0) != cudaSuccess)
            return fail(CJ_ERR_CUDA, "grouped plan: join failed");
    }
    return CJ_OK;
}

// Generate, request (compile in the background, or inline in sync mode) and
// ticket the plan's dispatcher.  `items` is the plan's work list on the host
// ({offset, T, 0} per item, groups contiguous, each ordered by T descending).
constexpr int kDispatchBlock = 256;

// The dispatcher's source for `minb` resident blocks per SM (the launch
// bounds' register cap), and its shared-memory need.
// A dispatcher variant: resident blocks per SM the launch bounds must allow
// (the register cap), the tile rule and the block size.
struct DispVariant {
    int minb, rule, block = kDispatchBlock;
};

// Shared memory a chunk of variant v may take: what minb blocks can hold
// together on one SM (228 KiB, less per block the 1 KiB the hardware
// reserves and 4 KiB for the dispatcher's static shared memory: 3,088
// bytes of chunk bookkeeping), at most 160 KiB.
long dispatch_smem_cap(DispVariant v) {
    return std::min<long>(160 * 1024, 233472 / v.minb - 5120);
}

std::string dispatcher_source(const cj_group_plan_s *p, DispVariant v, long *smem_out) {
    const int minb = v.minb;
    const int kBlock = v.block;
    const char *ct = p->dtype == CJ_F64 ? "double" : "float";
    std::string src = "#include \"update_chain.cuh\"\nnamespace cj {\n__global__ void __launch_bounds__(" +
                      std::to_string(kBlock) + ", " + std::to_string(minb) +
                      ")\nplan_dispatch(const long long* __restrict__ tickets, int n_tickets, "
                      "const long long* __restrict__ items, const " + std::string(ct) + "* __restrict__ A, " + ct +
                      "* __restrict__ X, int* __restrict__ counter) {\n"
                      "    dispatch_tickets<" + ct + ">(tickets, n_tickets, items, counter,\n"
                      "        [&](int g, const long long* it, int ninst, " + ct + "* sA, long long* so, int* ss) {\n"
                      "        switch (g) {\n";
    long smem = 0;
    for (size_t g = 0; g < p->groups.size(); ++g) {
        const auto &gr = p->groups[g];
        const int gdt = (p->dtype == CJ_BF16 && gr.n < 16) ? CJ_F32 : p->dtype;
        const auto t = dispatch_tile(gdt, gr.n, kBlock, v.rule, dispatch_smem_cap(v));
        smem = std::max(smem, cjg::chain_smem(gr.n, t[0], t[1], esize(gdt)));
        src += "        case " + std::to_string(g) + ": grouped_chunk_call<" + ct + ", " + std::to_string(gr.n) +
               ", " + std::to_string(t[0]) + ", " + std::to_string(t[1]) + ", " + std::to_string(kBlock) +
               ">(it, ninst, A, X, sA, so, ss); break;\n";
    }
    src += "        default: break;\n        }\n    });\n}\n}  // namespace cj\n";
    *smem_out = smem;
    return src;
}

// Request (compile in the background) a dispatcher variant; identical plans
// share it.
cj_handle_s *request_dispatcher(const cj_group_plan_s *p, DispVariant v) {
    long smem = 0;
    const std::string src = dispatcher_source(p, v, &smem);
    const std::string ks = "dispatch:" + src;
    std::lock_guard<std::mutex> lk(G.mu);
    auto it = G.cache.find(ks);
    if (it != G.cache.end()) return it->second;
    auto *h = new cj_handle_s();
    h->kernel = kDispatchKernel;
    h->a.dtype = p->dtype;
    h->a.tile[0] = v.block;
    h->a.tile[1] = (int)smem;
    h->a.tile[2] = v.minb;
    h->a.tile[3] = v.rule;
    h->custom_src = src;
    h->name_expr = "cj::plan_dispatch";
    h->impl.store(&h->generic, std::memory_order_release);   // no stand-in of its own
    h->state = ST_PENDING;
    // compiled on the background threads even in sync mode: the per-group
    // kernels serve until it is ready (cj_group_plan_wait)
    G.queue.push_back(h);
    G.qcv.notify_one();
    G.cache.emplace(ks, h);
    return h;
}

// Dispatcher variants: the first is requested at plan creation, the others
// by the plan's autotuner.  FP32 bodies fit 128 registers (two blocks of 256
// threads) without spilling and 80 (three) with small spills in the n < 8
// bodies; BF16 tensor-core bodies want more; FP64 rows of X need up to 255.
// FP32 starts with tile rule 1 (4 x 8 register blocks for n >= 16: 1.18 ms
// against 1.39 ms for rule 0 on the 10,000-instance batch) and also tries
// rule 0.
// BF16 also tries blocks of 128 threads, three per SM (170 registers: the
// n = 64 panel bodies fit without spilling, 12 warps per SM).
std::vector<DispVariant> dispatcher_variants(int dtype) {
    if (dtype == CJ_F64) return {{1, 0}};
    if (dtype == CJ_F32) return {{2, 1}, {3, 1}, {2, 0}, {3, 0}};
    return {{2, 0}, {1, 0}, {3, 0, 128}};
}

// Ticket the plan's work for variant v (each ticket one chunk of one group,
// chunks as large as v's body for that group takes), upload the tickets and
// request v's kernel.
cj_status make_dispatch_form(cj_group_plan_s *p, DispVariant v, cj_group_plan_s::DispForm *out) {
    struct Tk {
        double cost;
        long long first;
        int group, count;
    };
    std::vector<Tk> tk;
    for (size_t g = 0; g < p->groups.size(); ++g) {
        const auto &gr = p->groups[g];
        const int gdt = (p->dtype == CJ_BF16 && gr.n < 16) ? CJ_F32 : p->dtype;
        const auto t = dispatch_tile(gdt, gr.n, v.block, v.rule, dispatch_smem_cap(v));
        const double per = 2.0 * gr.n * gr.n * gr.n + 2.0 * gr.n * gr.n;
        for (int64_t c = 0; c < gr.n_items; c += t[1]) {
            Tk k{0.0, gr.first_item + c, (int)g, (int)std::min<int64_t>(t[1], gr.n_items - c)};
            for (int i = 0; i < k.count; ++i) k.cost += per * (double)p->h_items[3 * (k.first + i) + 1];
            tk.push_back(k);
        }
    }
    // longest chunks first
    std::stable_sort(tk.begin(), tk.end(), [](const Tk &x, const Tk &y) { return x.cost > y.cost; });
    std::vector<long long> host(2 * tk.size());
    for (size_t i = 0; i < tk.size(); ++i) {
        host[2 * i] = tk[i].first;
        host[2 * i + 1] = ((long long)tk[i].group << 16) | tk[i].count;
    }
    out->n_tickets = (int)tk.size();
    if (cudaMalloc(&out->d_tickets, sizeof(long long) * host.size()) != cudaSuccess)
        return fail(CJ_ERR_OOM, "grouped plan: dispatcher tickets");
    if (cudaMemcpy(out->d_tickets, host.data(), sizeof(long long) * host.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return fail(CJ_ERR_CUDA, "grouped plan: dispatcher ticket upload failed");
    out->h = request_dispatcher(p, v);
    return CJ_OK;
}

void use_dispatch_form(cj_group_plan_s *p, const cj_group_plan_s::DispForm &f) {
    p->disp = f.h;
    p->d_tickets = f.d_tickets;
    p->n_tickets = f.n_tickets;
}

// The plan's first dispatcher variant, requested at plan creation.  `items`
// is the plan's work list on the host ({offset, T, 0} per item, groups
// contiguous, each ordered by T descending).
cj_status plan_dispatcher(cj_group_plan_s *p, const std::vector<long long> &items) {
    p->h_items = items;
    cj_group_plan_s::DispForm f;
    const cj_status rc = make_dispatch_form(p, dispatcher_variants(p->dtype)[0], &f);
    p->disp_forms.push_back(f);   // freed with the plan even if the upload failed
    if (rc != CJ_OK) return rc;
    use_dispatch_form(p, f);
    return CJ_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
CJ_API cj_status cj_init(const cj_config *cfg, int device) {
    std::lock_guard<std::mutex> ilk(g_init_mu);
    if (G.inited) {
        if (device != G.device) return fail(CJ_ERR_INVALID_ARG, "already initialised for device %d", G.device);
        return CJ_OK;
    }
    cj_config c{};
    c.compile_threads = 1;
    c.enable_aot_set = 1;
    if (cfg) c = *cfg;
    if (c.compile_threads == 0) c.compile_threads = 1;
    if (c.compile_threads > 16) return fail(CJ_ERR_INVALID_ARG, "compile_threads must be <= 16");
    G.cfg = c;
    G.compile_only = (c.flags & CJ_CFG_COMPILE_ONLY) != 0;
    G.device = device;
    if (!G.compile_only) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            return fail(CJ_ERR_NO_DEVICE, "no CUDA device or driver");
        }
        if (device < 0 || device >= ndev) return fail(CJ_ERR_INVALID_ARG, "device %d out of range", device);
        int maj = 0, min = 0;
        cudaSetDevice(device);
        cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, device);
        cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, device);
        if (maj != 10 || min != 3)
            return fail(CJ_ERR_UNSUPPORTED_ARCH, "device is sm_%d%d; this library targets sm_103a", maj, min);
        if (cudaFree(nullptr) != cudaSuccess) return fail(CJ_ERR_CUDA, "could not create the device context");
        if (!load_driver()) return fail(CJ_ERR_NO_DEVICE, "driver entry points unavailable");
        cudaDeviceGetAttribute(&G.num_sms, cudaDevAttrMultiProcessorCount, device);
        cudaDeviceGetAttribute(&G.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        auto prep = [](const void *sym, CUfunction *out) -> bool {
            cudaFunction_t f = nullptr;
            if (cudaGetFuncBySymbol(&f, sym) != cudaSuccess) return false;
            *out = reinterpret_cast<CUfunction>(f);
            int stat = 0;
            drv.FuncGetAttribute(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, *out);
            return drv.FuncSetAttribute(*out, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                        G.smem_optin - stat) == CUDA_SUCCESS;
        };
        const auto &gk = cjint::generic_kernels();
        for (int d = 0; d < 2; ++d)
            if (!prep(gk.chain[d], &G.gen_chain[d]) || !prep(gk.ltimes[d], &G.gen_lt[d]) ||
                !prep(gk.grouped[d], &G.gen_grp[d]) || !prep(gk.eigen[d], &G.gen_eig[d]) ||
                !prep(gk.mass[d], &G.gen_mass[d]))
                return fail(CJ_ERR_CUDA, "could not load the generic kernels");
        int na = 0;
        const cjint::AotKernel *tab = cjint::aot_table(&na);
        G.aot.clear();
        for (int i = 0; i < na; ++i) {
            CUfunction f = nullptr;
            if (!prep(tab[i].fn, &f)) return fail(CJ_ERR_CUDA, "could not load AoT kernel %d", i);
            G.aot.push_back({tab[i], f});
        }
    } else {
        int na = 0;
        const cjint::AotKernel *tab = cjint::aot_table(&na);
        G.aot.clear();
        for (int i = 0; i < na; ++i) G.aot.push_back({tab[i], nullptr});
    }
    // Warm NVRTC here so that later compiles do no first-use work.
    CompileOut w = nvrtc_compile("#include \"update_chain.cuh\"\n__global__ void cj_warm() {}\n", nullptr);
    if (w.rc != NVRTC_SUCCESS) return fail(CJ_ERR_COMPILE, "NVRTC warm-up failed: %s", w.log.c_str());
    G.stop = false;
    G.requests = G.hits = G.ok = G.failed = G.aot_hits = 0;
    G.l_gen = G.l_aot = G.l_jit = G.l_tma = G.l_tma_fb = G.l_disp = 0;
    {
        std::lock_guard<std::mutex> lk(G.smu);
        G.compile_ms.clear();
        G.lookup_ns.clear();
        G.lookup_pos = 0;
    }
    static std::once_flag exit_hook;
    std::call_once(exit_hook, [] { std::atexit(stop_workers_at_exit); });
    for (uint32_t i = 0; i < c.compile_threads; ++i) G.workers.emplace_back(worker_loop);
    G.inited = true;
    t_err.clear();
    return CJ_OK;
}

CJ_API cj_status cj_specialize(cj_kernel_id k, const cj_template_args *req, cj_handle *out) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!req || !out) return fail(CJ_ERR_INVALID_ARG, "null argument");
    const auto t0 = clk::now();
    cj_template_args a;
    cj_status rc = validate_and_normalise((int)k, *req, a);
    if (rc != CJ_OK) return rc;
    unsigned char key[32];
    make_key((int)k, a, key);
    const std::string ks(reinterpret_cast<char *>(key), 32);
    cj_handle_s *h = nullptr;
    bool created = false;
    {
        std::lock_guard<std::mutex> lk(G.mu);
        G.requests++;
        auto it = G.cache.find(ks);
        if (it != G.cache.end()) {
            h = it->second;
            G.hits++;
        } else {
            h = new cj_handle_s();
            h->kernel = (int)k;
            h->a = a;
            memcpy(h->key, key, 32);
            generic_impl(h);
            h->impl.store(&h->generic, std::memory_order_release);
            created = true;
            if (a.flags & CJ_FLAG_GENERIC) {
                h->state = ST_GENERIC_ONLY;
            } else {
                const State::Aot *hit = nullptr;
                if (G.cfg.enable_aot_set && (int)k == CJ_K_UPDATE_CHAIN && !(a.flags & CJ_FLAG_NO_AOT) &&
                    !(a.flags & CJ_FLAG_INJECT_COMPILE_ERROR))
                    hit = find_aot(h);
                if (hit) {
                    h->spec.fn = hit->fn;
                    spec_geometry(h, h->spec);
                    h->spec.variant = V_AOT;
                    h->impl.store(&h->spec, std::memory_order_release);
                    h->state = ST_READY;
                    G.aot_hits++;
                } else {
                    h->name_expr = name_expression(h);
                    h->name_expr2 = fallback_name_expression(h);
                    h->state = ST_PENDING;
                    if (!G.cfg.sync) {
                        G.queue.push_back(h);
                        G.qcv.notify_one();
                    }
                }
            }
            G.cache.emplace(ks, h);
        }
    }
    *out = h;
    if (!created) {
        const double ns = std::chrono::duration<double, std::nano>(clk::now() - t0).count();
        std::lock_guard<std::mutex> lk(G.smu);
        if (G.lookup_ns.size() < 4096) G.lookup_ns.push_back(ns);
        else G.lookup_ns[G.lookup_pos++ % 4096] = ns;
    }
    if (G.cfg.sync) {
        if (created && h->state.load() == ST_PENDING) return compile_handle(h);
        std::unique_lock<std::mutex> lk(h->mu);
        h->cv.wait(lk, [h] { return h->state.load() != ST_PENDING; });
        if (h->state.load() == ST_FAILED) return fail(CJ_ERR_COMPILE, "%s", h->error.c_str());
    }
    return CJ_OK;
}

CJ_API cj_status cj_specialize_wait(cj_handle h, int timeout_ms) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!h) return fail(CJ_ERR_INVALID_ARG, "null handle");
    std::unique_lock<std::mutex> lk(h->mu);
    auto done = [h] { return h->state.load() != ST_PENDING; };
    if (timeout_ms < 0) h->cv.wait(lk, done);
    else if (!h->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return fail(CJ_ERR_TIMEOUT, "instantiation still compiling");
    if (h->state.load() == ST_FAILED) return fail(CJ_ERR_COMPILE, "%s", h->error.c_str());
    return CJ_OK;
}

// TMA tensor map of the (D, G, Z) tensor `in` in storage order lin, box (32
// directions, tg, tz): dimensions innermost first, row strides in bytes, a
// 128-byte swizzle when d is innermost (its 128-byte box rows), zero fill
// outside the tensor.  False when no map is possible: `in` not 16-byte
// aligned, or the innermost extent or box extent not a multiple of 4 floats
// (row strides and box starts must be 16-byte multiples).
bool lt_tensor_map(CUtensorMap *m, const void *in, int lin, long long D, long long G, long long Z, int tg, int tz) {
    const long long ext[3] = {D, G, Z};
    const int box[3] = {32, tg, tz};
    const int a2 = lt_axis_host(lin, 2), a1 = lt_axis_host(lin, 1), a0 = lt_axis_host(lin, 0);
    if (reinterpret_cast<uintptr_t>(in) % 16 || ext[a2] % 4 || box[a2] % 4) return false;
    for (long long e : ext)
        if (e > 0xFFFFFFFFll) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ext[a2], (cuuint64_t)ext[a1], (cuuint64_t)ext[a0]};
    const cuuint64_t strides[2] = {(cuuint64_t)ext[a2] * 4, (cuuint64_t)(ext[a2] * ext[a1]) * 4};
    const cuuint32_t bx[3] = {(cuuint32_t)box[a2], (cuuint32_t)box[a1], (cuuint32_t)box[a0]};
    const cuuint32_t es[3] = {1, 1, 1};
    return drv.TensorMapEncodeTiled(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(in), dims, strides, bx, es,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    a2 == 0 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

CJ_API cj_status cj_launch(cj_handle h, void *const *args, int64_t batch, void *cuda_stream) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!h || !args || batch < 0) return fail(CJ_ERR_INVALID_ARG, "null handle/args or negative batch");
    for (int i = 0; i < (is_lt(h->kernel) ? 5 : h->kernel == CJ_K_UPDATE_CHAIN ? 3 : 4); ++i)   // Eigen: 4
        if (!args[i]) return fail(CJ_ERR_INVALID_ARG, "argument %d is null", i);
    if (is_lt(h->kernel) && !(h->a.flags & CJ_FLAG_GENERIC) && ((h->a.tile[3] >> 16) & 0xf) >= 3) {
        // tile modes 3-6 move `in` and `out` in 16-byte vectors
        const uintptr_t in = reinterpret_cast<uintptr_t>(*reinterpret_cast<void *const *>(args[1]));
        const uintptr_t out = reinterpret_cast<uintptr_t>(*reinterpret_cast<void *const *>(args[2]));
        if ((in | out) & 15)
            return fail(CJ_ERR_INVALID_ARG, "tile modes 3-6 need 16-byte aligned in and out tensors");
    }
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "library initialised in compile-only mode");
    const Impl *im = h->impl.load(std::memory_order_acquire);
    const cj_template_args &a = h->a;
    CUstream st = reinterpret_cast<CUstream>(cuda_stream);
    CUresult r = CUDA_SUCCESS;
    if (h->kernel == CJ_K_UPDATE_CHAIN) {
        void *A = *reinterpret_cast<void *const *>(args[0]);
        void *X = *reinterpret_cast<void *const *>(args[1]);
        int steps = *reinterpret_cast<const int32_t *>(args[2]);
        if (!A || !X || steps < 1) return fail(CJ_ERR_INVALID_ARG, "null A/X or T < 1");
        if (batch == 0) return CJ_OK;
        long long b = batch;
        double c = 1.0 / ((double)a.n * (double)steps);
        // a batch whose full blocks would leave SMs idle is spread over up to
        // one block per SM, each taking fewer instances than it is shaped for
        int ipb = im->ipb;
        if (batch < (long long)ipb * G.num_sms) ipb = (int)std::max<long long>(1, (batch + G.num_sms - 1) / G.num_sms);
        unsigned grid = (unsigned)((batch + ipb - 1) / ipb);
        if (im->variant != V_GENERIC && a.tile[0] == 7)   // persistent: blocks keep their tensor memory
            grid = (unsigned)std::min<long long>(batch, (long long)G.num_sms * im->blocks_per_sm);
        if (im->variant == V_GENERIC) {
            int n = a.n, lay = a.layout_a;
            void *p[] = {&A, &X, &b, &steps, &c, &n, &lay, &ipb};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        } else {
            void *p[] = {&A, &X, &b, &steps, &c, &ipb};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        }
    } else if (is_mass(h->kernel)) {
        void *B1 = *reinterpret_cast<void *const *>(args[0]);
        void *op = *reinterpret_cast<void *const *>(args[1]);
        void *xv = *reinterpret_cast<void *const *>(args[2]);
        void *yv = *reinterpret_cast<void *const *>(args[3]);
        if (!B1 || !op || !xv || !yv) return fail(CJ_ERR_INVALID_ARG, "null B1/op/x/y");
        if (batch == 0) return CJ_OK;
        long long ne = batch;
        const long long groups = (batch + im->ipb - 1) / im->ipb;
        // the persistent kernel (tile[1] = 1): at most its resident blocks
        const unsigned grid = (unsigned)(im->variant != V_GENERIC && a.tile[1] == 1
                                             ? std::min(groups, (long long)G.num_sms * im->blocks_per_sm)
                                             : groups);
        if (im->variant == V_GENERIC) {
            int dim = a.d, D = a.n, Q = a.m, epb = im->ipb;
            void *p[] = {&B1, &op, &xv, &yv, &ne, &dim, &D, &Q, &epb};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        } else {
            void *p[] = {&B1, &op, &xv, &yv, &ne};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        }
    } else if (is_eig(h->kernel)) {
        void *M0 = *reinterpret_cast<void *const *>(args[0]);
        void *M = *reinterpret_cast<void *const *>(args[1]);
        int rep = *reinterpret_cast<const int32_t *>(args[2]);
        double c = *reinterpret_cast<const double *>(args[3]);
        if (!M0 || !M || rep < 0) return fail(CJ_ERR_INVALID_ARG, "null M0/M or negative repeat");
        if (batch == 0) return CJ_OK;
        long long b = batch;
        const unsigned grid = (unsigned)((batch + im->ipb - 1) / im->ipb);
        if (im->variant == V_GENERIC) {
            int n = a.n, ipb = im->ipb;
            void *p[] = {&M0, &M, &b, &rep, &c, &n, &ipb};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        } else {
            void *p[] = {&M0, &M, &b, &rep, &c};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        }
    } else if (is_lt(h->kernel)) {
        const LtView v = lt_view(h->kernel, a);
        void *L = *reinterpret_cast<void *const *>(args[0]);
        void *in = *reinterpret_cast<void *const *>(args[1]);
        void *out = *reinterpret_cast<void *const *>(args[2]);
        long long Gx = *reinterpret_cast<const int64_t *>(args[3]);
        long long Zx = *reinterpret_cast<const int64_t *>(args[4]);
        if (!L || !in || !out || Gx < 0 || Zx < 0) return fail(CJ_ERR_INVALID_ARG, "null tensor or negative G/Z");
        if (Gx == 0 || Zx == 0) return CJ_OK;
        if (im->variant == V_GENERIC) {
            int M = v.m, D = v.d, acc = v.acc;
            auto strides = [&](int lay, long long ex, long long *s) {
                // s[axis] for axis 0 = x, 1 = g, 2 = z
                const long long e[3] = {ex, Gx, Zx};
                static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                const int *o = order[lay];
                s[o[2]] = 1;
                s[o[1]] = e[o[2]];
                s[o[0]] = e[o[2]] * e[o[1]];
            };
            long long si[3], so[3];
            strides(v.lin, D, si);
            strides(v.lout, M, so);
            const long long cols = Gx * Zx;
            const unsigned grid = (unsigned)((cols + im->threads - 1) / im->threads);
            void *p[] = {&L, &in, &out, &Gx, &Zx, &M, &D, &si[0], &si[1], &si[2], &so[0], &so[1], &so[2], &acc};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        } else {
            const long long ntiles = ((Gx + a.tile[0] - 1) / a.tile[0]) * ((Zx + a.tile[1] - 1) / a.tile[1]);
            const int mode = (a.tile[3] >> 16) & 0xf;
            if (mode >= 4 && mode <= 6) {
                // tcgen05 kernels take a TMA tensor map of `in` (unused in mode 4); modes 5
                // and 6 fall back to their mode-4 twin when `in` admits none
                CUtensorMap map;
                memset(&map, 0, sizeof map);
                CUfunction fn = im->fn;
                int threads = im->threads, bps = im->blocks_per_sm;
                size_t smem = im->smem;
                const bool tma = mode >= 5 && lt_tensor_map(&map, in, v.lin, v.d, Gx, Zx, a.tile[0], a.tile[1]);
                if (mode >= 5 && !tma) {
                    fn = im->fn2;
                    threads = im->threads2;
                    smem = im->smem2;
                    bps = im->blocks2;
                }
                if (mode >= 5) (tma ? G.l_tma : G.l_tma_fb)++;
                const unsigned grid = (unsigned)std::min(ntiles, (long long)G.num_sms * bps);
                void *p[] = {&L, &in, &out, &Gx, &Zx, &map};
                r = drv.LaunchKernel(fn, grid, 1, 1, threads, 1, 1, (unsigned)smem, st, p, nullptr);
            } else {
                const long long cap = (long long)G.num_sms * im->blocks_per_sm;
                const unsigned grid = (unsigned)std::min(ntiles, cap);
                void *p[] = {&L, &in, &out, &Gx, &Zx};
                r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
            }
        }
    } else {
        void *items = *reinterpret_cast<void *const *>(args[0]);
        void *A = *reinterpret_cast<void *const *>(args[1]);
        void *X = *reinterpret_cast<void *const *>(args[2]);
        void *counter = *reinterpret_cast<void *const *>(args[3]);
        if (!items || !A || !X || !counter) return fail(CJ_ERR_INVALID_ARG, "null worklist/pool/counter");
        if (batch == 0) return CJ_OK;
        long long ni = batch;
        const long long chunks = (batch + im->ipb - 1) / im->ipb;
        const unsigned grid = (unsigned)std::min(chunks, (long long)G.num_sms * im->blocks_per_sm);
        if (im->variant == V_GENERIC) {
            int n = a.n, ipb = im->ipb;
            void *p[] = {&items, &A, &X, &counter, &ni, &n, &ipb};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        } else {
            void *p[] = {&items, &A, &X, &counter, &ni};
            r = drv.LaunchKernel(im->fn, grid, 1, 1, im->threads, 1, 1, (unsigned)im->smem, st, p, nullptr);
        }
    }
    if (r != CUDA_SUCCESS) return fail(CJ_ERR_CUDA, "launch failed: %s", cu_str(r));
    (im->variant == V_GENERIC ? G.l_gen : im->variant == V_AOT ? G.l_aot : G.l_jit)++;
    return CJ_OK;
}

CJ_API cj_status cj_stats(cj_stats_t *out) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!out) return fail(CJ_ERR_INVALID_ARG, "null output");
    out->requests = G.requests;
    out->cache_hits = G.hits;
    out->compiles_ok = G.ok;
    out->compiles_failed = G.failed;
    out->aot_hits = G.aot_hits;
    out->launches_generic = G.l_gen;
    out->launches_aot = G.l_aot;
    out->launches_jit = G.l_jit;
    out->launches_tma = G.l_tma;
    out->launches_tma_fallback = G.l_tma_fb;
    out->launches_dispatch = G.l_disp;
    {
        std::lock_guard<std::mutex> lk(G.smu);
        out->compile_ms_p50 = percentile(G.compile_ms, 0.5);
        out->compile_ms_p95 = percentile(G.compile_ms, 0.95);
        out->lookup_ns_p50 = percentile(G.lookup_ns, 0.5);
    }
    // expired bounded waits: the counters of every module that has them,
    // read after all queued work has finished
    out->wait_timeouts = 0;
    if (G.compile_only) return CJ_OK;
    std::vector<CUdeviceptr> counters;
    {
        std::lock_guard<std::mutex> lk(G.mu);
        for (const auto &kv : G.cache)
            if (kv.second->state.load(std::memory_order_acquire) == ST_READY && kv.second->wait_count)
                counters.push_back(kv.second->wait_count);
    }
    if (counters.empty()) return CJ_OK;
    if (cudaDeviceSynchronize() != cudaSuccess)
        return fail(CJ_ERR_CUDA, "cj_stats: device synchronize failed: %s", cudaGetErrorString(cudaGetLastError()));
    for (CUdeviceptr p : counters) {
        uint32_t c = 0;
        if (cudaMemcpy(&c, reinterpret_cast<void *>(p), sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(CJ_ERR_CUDA, "cj_stats: reading a wait-timeout counter failed");
        out->wait_timeouts += c;
    }
    return CJ_OK;
}

CJ_API cj_status cj_handle_info(cj_handle h, char *key_hex, size_t cap, int *variant) {
    if (!h) return fail(CJ_ERR_INVALID_ARG, "null handle");
    if (key_hex) {
        if (cap < 65) return fail(CJ_ERR_INVALID_ARG, "key buffer needs 65 bytes");
        for (int i = 0; i < 32; ++i) snprintf(key_hex + 2 * i, 3, "%02x", h->key[i]);
    }
    if (variant) {
        const Impl *im = h->impl.load(std::memory_order_acquire);
        if (G.compile_only) {
            const int s = h->state.load();
            *variant = h->spec.variant == V_AOT ? V_AOT : (s == ST_READY ? V_JIT : V_GENERIC);
        } else {
            *variant = im->variant;
        }
    }
    return CJ_OK;
}

CJ_API cj_status cj_handle_regs(cj_handle h, int *regs, int *static_smem) {
    if (!h) return fail(CJ_ERR_INVALID_ARG, "null handle");
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    const Impl *im = h->impl.load(std::memory_order_acquire);
    if (regs && drv.FuncGetAttribute(regs, CU_FUNC_ATTRIBUTE_NUM_REGS, im->fn) != CUDA_SUCCESS)
        return fail(CJ_ERR_CUDA, "cuFuncGetAttribute failed");
    if (static_smem && drv.FuncGetAttribute(static_smem, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, im->fn) != CUDA_SUCCESS)
        return fail(CJ_ERR_CUDA, "cuFuncGetAttribute failed");
    return CJ_OK;
}

CJ_API cj_status cj_handle_wait_timeouts(cj_handle h, uint32_t *count, int reset) {
    if (!h || !count) return fail(CJ_ERR_INVALID_ARG, "null handle or count");
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    *count = 0;
    // no JIT module (AoT or generic kernels), or a module without bounded waits
    if (h->state.load(std::memory_order_acquire) != ST_READY || !h->wait_count) return CJ_OK;
    const CUdeviceptr p = h->wait_count;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(count, reinterpret_cast<void *>(p), sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (reset && cudaMemset(reinterpret_cast<void *>(p), 0, sizeof(uint32_t)) != cudaSuccess))
        return fail(CJ_ERR_CUDA, "reading the wait-timeout counter failed");
    return CJ_OK;
}

CJ_API cj_status cj_group_plan_create(int32_t dtype, int64_t count, const int32_t *n, const int32_t *steps,
                                      uint32_t flags, cj_group_plan *out) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    if (!out || count < 0 || (count > 0 && (!n || !steps)))
        return fail(CJ_ERR_INVALID_ARG, "null output or inputs");
    if (dtype != CJ_F64 && dtype != CJ_F32 && dtype != CJ_BF16)
        return fail(CJ_ERR_INVALID_ARG, "grouped plans support f64, f32 and bf16");
    if (flags & ~CJ_FLAG_GENERIC) return fail(CJ_ERR_INVALID_ARG, "grouped plans accept only CJ_FLAG_GENERIC");
    for (int64_t k = 0; k < count; ++k)
        if (n[k] < 1 || n[k] > 64 || steps[k] < 1) return fail(CJ_ERR_INVALID_ARG, "instance %lld out of range", (long long)k);
    auto *p = new cj_group_plan_s();
    p->dtype = dtype;
    p->count = count;
    std::vector<int64_t> off(count);
    int64_t acc = 0;
    for (int64_t k = 0; k < count; ++k) {
        off[k] = acc;
        acc += (int64_t)n[k] * n[k];
    }
    p->pool_elems = acc;
    // group by n; items ordered by T descending (ties by index)
    std::vector<std::vector<int64_t>> by_n(65);
    for (int64_t k = 0; k < count; ++k) by_n[n[k]].push_back(k);
    std::vector<long long> items;
    for (int nn = 1; nn <= 64; ++nn) {
        auto &v = by_n[nn];
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [&](int64_t x, int64_t y) { return steps[x] > steps[y]; });
        cj_group_plan_s::Group g;
        g.n = nn;
        g.first_item = (int64_t)items.size() / 3;
        g.n_items = (int64_t)v.size();
        for (int64_t k : v) {
            items.push_back(off[k]);
            items.push_back(steps[k]);
            items.push_back(0);
            g.cost += (double)steps[k] * nn * nn * nn;
        }
        p->groups.push_back(g);
    }
    // the most expensive groups are launched first
    std::stable_sort(p->groups.begin(), p->groups.end(),
                     [](const cj_group_plan_s::Group &x, const cj_group_plan_s::Group &y) { return x.cost > y.cost; });
    for (auto &g : p->groups) {
        cj_template_args a{};
        a.dtype = (dtype == CJ_BF16 && g.n < 16) ? CJ_F32 : dtype;   // bf16 runs n >= 16 on tensor cores
        a.n = g.n;
        a.flags = flags;
        cj_status rc = cj_specialize(CJ_K_UPDATE_CHAIN_GROUPED, &a, &g.h);
        if (rc != CJ_OK && rc != CJ_ERR_COMPILE) {
            plan_free(p);
            return rc;
        }
    }
    const size_t ng = p->groups.size() + 1;   // one counter per group, one for the dispatcher
    if (cudaMalloc(&p->d_counters, sizeof(int) * ng) != cudaSuccess ||
        (!items.empty() && cudaMalloc(&p->d_items, sizeof(long long) * items.size()) != cudaSuccess)) {
        plan_free(p);
        return fail(CJ_ERR_OOM, "grouped plan: device allocation failed");
    }
    if (!items.empty() &&
        cudaMemcpy(p->d_items, items.data(), sizeof(long long) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        plan_free(p);
        return fail(CJ_ERR_CUDA, "grouped plan: work list upload failed");
    }
    if (!(flags & CJ_FLAG_GENERIC) && !p->groups.empty()) {
        cj_status rc = plan_dispatcher(p, items);
        if (rc != CJ_OK && rc != CJ_ERR_COMPILE) {
            plan_free(p);
            return rc;
        }
    }
    const size_t ns = std::min<size_t>(64, std::max<size_t>(1, p->groups.size()));   // one stream per group
    p->streams.resize(ns);
    p->join.resize(ns);
    for (size_t i = 0; i < ns; ++i) {
        cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking);
    {
        std::lock_guard<std::mutex> lk(G.mu);
        G.plans.push_back(p);
    }
    *out = p;
    return CJ_OK;
}

namespace {
cj_status plan_launch(cj_group_plan_s *p, const void *A_pool, void *X_pool, cudaStream_t st, int use_graph);
}

CJ_API cj_status cj_group_plan_launch(cj_group_plan p, const void *A_pool, void *X_pool, void *cuda_stream,
                                      int use_graph) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!p || (p->pool_elems > 0 && (!A_pool || !X_pool))) return fail(CJ_ERR_INVALID_ARG, "null plan or pool");
    if (p->groups.empty()) return CJ_OK;
    if (use_graph & ~(CJ_PLAN_GRAPH | CJ_PLAN_PER_GROUP)) return fail(CJ_ERR_INVALID_ARG, "unknown launch flags");
    return plan_launch(p, A_pool, X_pool, reinterpret_cast<cudaStream_t>(cuda_stream), use_graph);
}

namespace {
// cj_group_plan_launch after argument checks (also used by the autotuner).
cj_status plan_launch(cj_group_plan_s *p, const void *A_pool, void *X_pool, cudaStream_t st, int use_graph) {
    const bool per_group = (use_graph & CJ_PLAN_PER_GROUP) != 0;
    if (!(use_graph & CJ_PLAN_GRAPH)) return plan_record(p, A_pool, X_pool, st, per_group);
    // what the captured graph launches: the dispatcher, or every group's kernel
    std::vector<const void *> impls;
    if (!per_group && p->use_dispatcher && dispatcher_ready(p))
        impls.push_back(p->disp->impl.load(std::memory_order_acquire));
    else
        for (auto &g : p->groups) impls.push_back(g.h->impl.load(std::memory_order_acquire));
    if (!p->exec || p->g_A != A_pool || p->g_X != X_pool || p->g_impls != impls) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        p->exec = nullptr;
        p->graph = nullptr;
        if (cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(CJ_ERR_CUDA, "stream capture could not start");
        cj_status rc = plan_record(p, A_pool, X_pool, p->capture, per_group);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->capture, &g);
        if (rc != CJ_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess || cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(CJ_ERR_CUDA, "graph capture/instantiate failed");
        }
        p->graph = g;
        p->g_A = A_pool;
        p->g_X = X_pool;
        p->g_impls = impls;
    }
    if (cudaGraphLaunch(p->exec, st) != cudaSuccess) return fail(CJ_ERR_CUDA, "graph launch failed");
    return CJ_OK;
}
}  // namespace

CJ_API cj_status cj_group_plan_autotune(cj_group_plan p, const void *A_pool, void *X_pool, void *cuda_stream,
                                        int32_t max_groups, int32_t reps, int32_t *changed) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    if (!p || (p->pool_elems > 0 && (!A_pool || !X_pool)) || max_groups < 0)
        return fail(CJ_ERR_INVALID_ARG, "null plan or pool, or negative group count");
    if (reps < 1) reps = 3;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t ng = max_groups > 0 ? std::min<size_t>((size_t)max_groups, p->groups.size()) : p->groups.size();
    int nchg = 0;
    // 0. the dispatcher's other variants start compiling now, beside the groups' candidates
    if (p->disp) {
        const std::vector<DispVariant> vs = dispatcher_variants(p->dtype);
        for (size_t i = p->disp_forms.size(); i < vs.size(); ++i) {
            cj_group_plan_s::DispForm f;
            const cj_status rf = make_dispatch_form(p, vs[i], &f);
            if (rf != CJ_OK) {
                if (f.d_tickets) cudaFree(f.d_tickets);
                return rf;
            }
            p->disp_forms.push_back(f);
        }
    }
    // 1. request every candidate tile of the tuned groups (the most expensive
    //    first: groups are kept sorted by cost); in async mode they compile in
    //    parallel on the background threads
    std::vector<std::vector<cj_handle>> cand(ng);
    for (size_t g = 0; g < ng; ++g) {
        cj_template_args a{};
        a.dtype = (p->dtype == CJ_BF16 && p->groups[g].n < 16) ? CJ_F32 : p->dtype;
        a.n = p->groups[g].n;
        int32_t tiles[4 * 32], cnt = 0;
        if (cj_candidates(CJ_K_UPDATE_CHAIN_GROUPED, &a, tiles, 32, &cnt) != CJ_OK) continue;
        for (int32_t c = 0; c < std::min<int32_t>(cnt, 32); ++c) {
            if (tiles[4 * c + 1] > 256) continue;   // grouped chunks hold at most 256 instances
            cj_template_args t = a;
            for (int i = 0; i < 4; ++i) t.tile[i] = tiles[4 * c + i];
            cj_handle h = nullptr;
            if (cj_specialize(CJ_K_UPDATE_CHAIN_GROUPED, &t, &h) == CJ_OK) cand[g].push_back(h);
        }
    }
    // 2. time each compiled candidate on the group's own work list (counter
    //    reset before every launch; each launch writes correct X for the group)
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(CJ_ERR_CUDA, "event creation failed");
    cj_status rc = CJ_OK;
    for (size_t g = 0; g < ng && rc == CJ_OK; ++g) {
        auto &gr = p->groups[g];
        void *items = p->d_items + 3 * gr.first_item;
        void *counter = p->d_counters + g;
        const void *a = A_pool;
        void *x = X_pool;
        void *args[4] = {&items, &a, &x, &counter};
        float best = 0;
        cj_handle best_h = nullptr;
        for (cj_handle h : cand[g]) {
            if (cj_specialize_wait(h, -1) != CJ_OK) continue;   // failed compiles are not candidates
            std::vector<float> ms;
            for (int r = 0; r <= reps && rc == CJ_OK; ++r) {    // r = 0 warms up
                if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess)
                    rc = fail(CJ_ERR_CUDA, "grouped autotune: memset/event failed");
                else if ((rc = cj_launch(h, args, gr.n_items, st)) == CJ_OK) {
                    float t = 0;
                    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                        rc = fail(CJ_ERR_CUDA, "grouped autotune: timing failed");
                    else if (r > 0)
                        ms.push_back(t);
                }
            }
            if (rc != CJ_OK) break;
            std::sort(ms.begin(), ms.end());
            const float med = ms[ms.size() / 2];
            if (!best_h || med < best) {
                best = med;
                best_h = h;
            }
        }
        if (best_h && best_h != gr.h) {
            gr.h = best_h;   // the next graph launch re-captures (the launch function changed)
            ++nchg;
        }
    }
    // 3. the launch form: every compiled dispatcher variant against one
    //    kernel per group with the tiles just chosen, each timed as a whole
    //    launch, as a CUDA graph and issued directly (a form's time is the
    //    faster of the two); the fastest is kept.
    //    A form's time is that of launches issued back to back, as a caller
    //    issues them in steady state: one warm-up launch (it captures the
    //    graph), then max(reps, 10) launches between two events.  Timing each
    //    launch with a host wait in between would add the host's submission
    //    of the launch to it, which is far larger for one kernel per group
    //    (tens of graph nodes or launches) than for the dispatcher.
    const int form_reps = std::max(reps, 10);
    auto time_form = [&](int flags, float *out) {
        float t = 0;
        if ((rc = plan_launch(p, A_pool, X_pool, st, flags)) != CJ_OK) return;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) {
            rc = fail(CJ_ERR_CUDA, "grouped autotune: event failed");
            return;
        }
        for (int r = 0; r < form_reps && rc == CJ_OK; ++r) rc = plan_launch(p, A_pool, X_pool, st, flags);
        if (rc != CJ_OK) return;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = fail(CJ_ERR_CUDA, "grouped autotune: timing failed");
            return;
        }
        *out = std::min(*out, t / form_reps);
    };
    if (rc == CJ_OK && !p->disp_forms.empty()) {
        float best_disp = INFINITY, best_group = INFINITY;
        cj_group_plan_s::DispForm best_f{p->disp, p->d_tickets, p->n_tickets};
        p->use_dispatcher = true;
        for (const auto &f : p->disp_forms) {
            if (rc != CJ_OK) break;
            if (cj_specialize_wait(f.h, -1) != CJ_OK) continue;   // a variant that failed to compile
            use_dispatch_form(p, f);
            if (!dispatcher_ready(p)) continue;
            float t = INFINITY;
            time_form(CJ_PLAN_GRAPH, &t);
            time_form(0, &t);
            if (t < best_disp) {
                best_disp = t;
                best_f = f;
            }
        }
        use_dispatch_form(p, best_f);
        time_form(CJ_PLAN_GRAPH | CJ_PLAN_PER_GROUP, &best_group);
        time_form(CJ_PLAN_PER_GROUP, &best_group);
        p->use_dispatcher = rc != CJ_OK || best_disp <= best_group;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (changed) *changed = nchg;
    return rc;
}

CJ_API cj_status cj_group_plan_wait(cj_group_plan p, int timeout_ms) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (!p) return fail(CJ_ERR_INVALID_ARG, "null plan");
    const auto end = clk::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    cj_status worst = CJ_OK;
    for (auto &g : p->groups) {
        int left = -1;
        if (timeout_ms >= 0)
            left = (int)std::max<long long>(
                0, std::chrono::duration_cast<std::chrono::milliseconds>(end - clk::now()).count());
        const cj_status rc = cj_specialize_wait(g.h, left);
        if (rc == CJ_ERR_TIMEOUT) return rc;
        if (rc != CJ_OK) worst = rc;
    }
    if (p->disp) {
        int left = -1;
        if (timeout_ms >= 0)
            left = (int)std::max<long long>(
                0, std::chrono::duration_cast<std::chrono::milliseconds>(end - clk::now()).count());
        const cj_status rc = cj_specialize_wait(p->disp, left);
        if (rc == CJ_ERR_TIMEOUT) return rc;
        if (rc != CJ_OK) return fail(rc, "the plan's dispatcher failed to compile (per-group kernels serve): %s",
                                     p->disp->error.c_str());
    }
    return worst == CJ_OK ? CJ_OK : fail(worst, "a group's instantiation failed to compile; it runs generic");
}

CJ_API cj_status cj_group_plan_dispatcher(cj_group_plan p, int32_t *state, int32_t *n_tickets, int32_t *threads,
                                          int32_t *blocks_per_sm) {
    if (!p) return fail(CJ_ERR_INVALID_ARG, "null plan");
    if (state) {
        const int s = p->disp ? p->disp->state.load(std::memory_order_acquire) : -1;
        *state = !p->disp ? 0 : s == ST_PENDING ? 1 : !dispatcher_ready(p) ? 3 : p->use_dispatcher ? 2 : 4;
    }
    if (n_tickets) *n_tickets = p->n_tickets;
    if (threads) *threads = p->disp ? p->disp->a.tile[0] : 0;
    if (blocks_per_sm) *blocks_per_sm = dispatcher_ready(p) ? p->disp->spec.blocks_per_sm : 0;
    return CJ_OK;
}

CJ_API cj_status cj_group_plan_use_dispatcher(cj_group_plan p, int32_t variant, int32_t *variants) {
    if (!p) return fail(CJ_ERR_INVALID_ARG, "null plan");
    const std::vector<DispVariant> vs = dispatcher_variants(p->dtype);
    if (variants) *variants = p->disp ? (int32_t)vs.size() : 0;
    if (variant < 0) return CJ_OK;
    if (!p->disp) return fail(CJ_ERR_INVALID_ARG, "plan has no dispatcher (CJ_FLAG_GENERIC)");
    if (variant >= (int32_t)vs.size()) return fail(CJ_ERR_INVALID_ARG, "dispatcher variant %d out of range", variant);
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    // forms are kept in the order of dispatcher_variants: create the missing ones up to `variant`
    for (size_t i = p->disp_forms.size(); i <= (size_t)variant; ++i) {
        cj_group_plan_s::DispForm f;
        const cj_status rf = make_dispatch_form(p, vs[i], &f);
        if (rf != CJ_OK) {
            if (f.d_tickets) cudaFree(f.d_tickets);
            return rf;
        }
        p->disp_forms.push_back(f);
    }
    const cj_group_plan_s::DispForm f = p->disp_forms[(size_t)variant];
    if (cj_specialize_wait(f.h, -1) != CJ_OK) return fail(CJ_ERR_COMPILE, "dispatcher variant %d failed to compile", variant);
    use_dispatch_form(p, f);
    p->use_dispatcher = true;
    return CJ_OK;
}

CJ_API cj_status cj_group_plan_info(cj_group_plan p, int32_t *n_groups, int64_t *pool_elems) {
    if (!p) return fail(CJ_ERR_INVALID_ARG, "null plan");
    if (n_groups) *n_groups = (int32_t)p->groups.size();
    if (pool_elems) *pool_elems = p->pool_elems;
    return CJ_OK;
}

CJ_API cj_status cj_group_plan_destroy(cj_group_plan p) {
    if (!p) return fail(CJ_ERR_INVALID_ARG, "null plan");
    {
        std::lock_guard<std::mutex> lk(G.mu);
        G.plans.erase(std::remove(G.plans.begin(), G.plans.end(), p), G.plans.end());
    }
    plan_free(p);
    return CJ_OK;
}

CJ_API cj_status cj_measure_fma_peak(int32_t dtype, int32_t tensor, void *cuda_stream, double *tflops) {
    if (!G.inited) return fail(CJ_ERR_NOT_INITIALIZED, "cj_init has not been called");
    if (G.compile_only) return fail(CJ_ERR_NO_DEVICE, "compile-only mode");
    if (!tflops || (dtype != CJ_F64 && dtype != CJ_F32) || (tensor && dtype != CJ_F64))
        return fail(CJ_ERR_INVALID_ARG, "dtype must be f64 or f32 (tensor: f64 only)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const void *k = tensor ? cjint::peak_dmma_kernel() : cjint::peak_fma_kernel(dtype);
    const unsigned grid = (unsigned)G.num_sms * 8u;
    int iters = tensor ? 1024 : dtype == CJ_F64 ? 4096 : 65536;
    double ad = 0.9999, bd = 1e-4;
    float af = 0.9999f, bf = 1e-4f;
    void *args_d[] = {&iters, &ad, &bd};
    void *args_f[] = {&iters, &af, &bf};
    void **args = dtype == CJ_F64 ? args_d : args_f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t err = cudaLaunchKernel(k, grid, 256, args, 0, st);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = cudaLaunchKernel(k, grid, 256, args, 0, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || ms <= 0) return fail(CJ_ERR_CUDA, "peak kernel failed: %s", cudaGetErrorString(err));
    // per thread and iteration: 8 FMA chains (2 flops each), or 8 mma.sync
    // m8n8k4 per warp (each 8 * 8 * 4 = 256 FMA = 512 flops, 16 per thread)
    const double per = tensor ? 8.0 * 16.0 : 8.0 * 2.0;
    const double flops = 3.0 * per * iters * (double)grid * 256.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return CJ_OK;
}

CJ_API const char *cj_last_error(void) { return t_err.c_str(); }

namespace cjint {
void set_last_error(const char *msg) { t_err = msg; }
void default_tile_of(int k, const cj_template_args &a, int tile_out[4]) {
    cj_template_args r = a;
    default_tile(k, r);
    for (int i = 0; i < 4; ++i) tile_out[i] = r.tile[i];
}
}  // namespace cjint

CJ_API cj_status cj_shutdown(void) {
    std::lock_guard<std::mutex> ilk(g_init_mu);
    if (!G.inited) return CJ_OK;
    {
        std::lock_guard<std::mutex> lk(G.mu);
        G.stop = true;
    }
    G.qcv.notify_all();
    for (auto &t : G.workers) t.join();
    G.workers.clear();
    if (!G.compile_only) cudaDeviceSynchronize();
    for (auto *p : G.plans) plan_free(p);
    G.plans.clear();
    for (auto &kv : G.cache) {
        cj_handle_s *h = kv.second;
        if (h->lib) drv.LibraryUnload(h->lib);
        delete h;
    }
    G.cache.clear();
    G.queue.clear();
    G.decisions.clear();
    cjint::noalloc_forget();
    G.inited = false;
    return CJ_OK;
}
