/*
 * cj.h -- C ABI of libcj: runtime template specialization of numeric CUDA
 * kernels for sm_103a (B300).
 *
 * The operation (ClangJIT, Finkel, Poliakoff and Richards, 2019): a function
 * template whose non-type template arguments (matrix size N, storage order)
 * and type arguments (dtype) become known only while the program runs is
 * instantiated and compiled at run time, cached in a program-global table
 * keyed on those arguments, and called through the result (Sec. 4,
 * Algorithm 1).  Compilation reads only data embedded in the running binary,
 * never the file system (Sec. 1 design requirement; Sec. 4 in-memory file
 * system).  Explicit specializations compiled ahead of time are used instead
 * of JIT compiling the same instantiation (Sec. 2).  Unlike the paper's
 * attribute, every call here has an error path and a fallback (Sec. 6,
 * critique of the attribute design): while an instantiation is compiling, or
 * if its compilation failed, launches run a generic runtime-N kernel.
 *
 * Kernels (all on the caller's stream, inputs and outputs in device memory
 * owned by the caller):
 *   CJ_K_UPDATE_CHAIN  -- per instance b: X_0 = I, X_{k+1} = X_k + c X_k A_b,
 *                         c = 1/(N T), k = 0..T-1, output X_T.  The paper's
 *                         Eigen benchmark loop (Sec. 5, Listings eigen1/eigen2)
 *                         in a stable form, batched over instances.
 *   CJ_K_LTIMES        -- out[m][g][z] = sum_d L[m][d] in[d][g][z], storage
 *                         orders of in and out chosen at run time (Kripke
 *                         LTimes, Sec. 5.2, Listings kripold/kripnew).
 *   CJ_K_LPLUSTIMES    -- the adjoint contraction named beside LTimes
 *                         (Sec. 5.2): in[d][g][z] += sum_m Lp[d][m] out[m][g][z].
 *   CJ_K_UPDATE_CHAIN_GROUPED -- the update chain over a work list of
 *                         instances of one size N but different step counts,
 *                         pulled by a persistent kernel (batch amortization of
 *                         the instantiation lookup, Sec. 5.1).
 *   CJ_K_EIGEN_RECURRENCE -- the Eigen benchmark's literal recurrence (Sec. 5,
 *                         Listing eigen1) batched: per instance
 *                         M_{k+1} = Ones + c (M_k + M_k M_k), k = 0..R-1, from a
 *                         caller-given M_0 (the listing: c = 5e-5, M_0(i, j) =
 *                         i + N j).  It grows without bound; compare over few
 *                         repeats.
 *   CJ_K_MASS          -- the mass operator of tensor-product finite elements
 *                         (the Laghos kernel of Sec. 5, specialized on the
 *                         dimension, dofs and quadrature points per
 *                         dimension): per element e, y_e = B^T diag(op_e) B x_e
 *                         with B the Kronecker product of the 1-D basis
 *                         matrix B1, evaluated by sum factorization.
 *
 * Thread safety: every function may be called from any host thread.
 * cj_specialize serialises on one mutex; cj_launch takes no lock.
 * Status: every function returns cj_status; cj_last_error() gives a
 * thread-local message (the NVRTC log after a compile failure).
 */
#ifndef CJ_H
#define CJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CJ_OK = 0,
    CJ_ERR_INVALID_ARG = 1,      /* bad argument; nothing was launched or changed */
    CJ_ERR_NOT_INITIALIZED = 2,  /* cj_init has not succeeded */
    CJ_ERR_NO_DEVICE = 3,        /* no CUDA device / driver (or compile-only mode on launch) */
    CJ_ERR_UNSUPPORTED_ARCH = 4, /* device is not compute capability 10.3 */
    CJ_ERR_COMPILE = 5,          /* NVRTC or module load failed; see cj_last_error */
    CJ_ERR_CUDA = 6,             /* a CUDA driver/runtime call failed */
    CJ_ERR_OOM = 7,              /* host or device allocation failed */
    CJ_ERR_TIMEOUT = 8,          /* cj_specialize_wait: still compiling */
    CJ_ERR_PENDING = 9           /* reserved */
} cj_status;

typedef enum {
    CJ_K_UPDATE_CHAIN = 1,
    CJ_K_LTIMES = 2,
    CJ_K_UPDATE_CHAIN_GROUPED = 3,
    CJ_K_LPLUSTIMES = 4,
    CJ_K_EIGEN_RECURRENCE = 5,
    CJ_K_MASS = 6
} cj_kernel_id;

typedef enum {
    CJ_F64 = 0,
    CJ_F32 = 1,
    CJ_BF16 = 2    /* bf16 tensor-core operands, fp32 accumulate, fp32 state; N >= 16 */
} cj_dtype;

/* Request flags (cj_template_args.flags). */
#define CJ_FLAG_GENERIC 0x1u      /* use the generic runtime-N kernel, never compile */
#define CJ_FLAG_NO_AOT 0x2u       /* JIT compile even where an AoT specialization exists */
#define CJ_FLAG_INJECT_COMPILE_ERROR 0x100u  /* test hook: submit a template that fails to compile */
/* test hook (LTimes tile modes 4-6 only): compile the tensor-core kernel
 * with producers that never signal a filled operand stage, so that every
 * block's bounded wait expires (about a second); blocks then stop and
 * cj_handle_wait_timeouts reports them, and `out` is left incomplete */
#define CJ_FLAG_INJECT_WAIT_TIMEOUT 0x200u

/* Config flags (cj_config.flags). */
#define CJ_CFG_COMPILE_ONLY 0x1u  /* no device: compile to CUBIN, never load or launch */

typedef struct {
    uint32_t sync;             /* 1: cj_specialize blocks until the instantiation is compiled */
    uint32_t compile_threads;  /* background compile threads (0 -> 1) */
    uint32_t use_cost_model;   /* 1: tile = 0 requests consult the loaded cost model */
    uint32_t enable_aot_set;   /* 1: N in {4,8,16,32} (f64/f32 update chain) use AoT kernels */
    uint32_t debug_bounds;     /* reserved */
    uint32_t flags;            /* CJ_CFG_* */
} cj_config;

/*
 * Runtime template arguments.  Unused fields must be 0 (they are ignored and
 * zeroed in the key).
 *   UPDATE_CHAIN:  dtype, n (1..64), layout_a (0 row-major, 1 column-major
 *                  storage of each A_b and X_b), tile.
 *   LTIMES:        dtype (f64/f32), layout_a = storage order of in, layout_b =
 *                  storage order of out, m (1..64), d (1..128), tile.
 *                  Storage orders list (x, g, z) slowest to fastest, x = d for
 *                  in and m for out: 0 XGZ, 1 XZG, 2 GXZ, 3 GZX, 4 ZXG, 5 ZGX.
 *   UPDATE_CHAIN_GROUPED: dtype, n (1..64), tile (row-major only).
 *   EIGEN_RECURRENCE: dtype (f64/f32), n (1..32), tile (row-major only).
 *   MASS:          dtype (f64/f32), d = dimension (2 or 3), n = dofs per
 *                  dimension D (1..16), m = quadrature points per dimension Q
 *                  (1..16): the paper's Laghos key (DIM << 16) | ((D - 1) << 8)
 *                  | (Q >> 1) in fields of its own; tile.
 *   LPLUSTIMES:    as LTIMES (layout_a = order of the accumulated `in`,
 *                  layout_b = order of the input `out`, m, d); the tile is
 *                  an LTimes tile of the swapped problem (d output rows, m
 *                  contracted, orders exchanged), defaults likewise.
 * tile = {0,0,0,0} means "choose": the cost model if enabled and loaded,
 * else the default rule below.  Meaning of tile fields:
 *   update chain: {mapping, instances per block, 0, 0}; mapping 1 = one thread
 *     per row of X (A staged in shared memory), 2 = one thread per instance
 *     (X and A in registers, n <= 8), 3 = bf16 tensor-core warp tile,
 *     4 = FP64 tensor cores (mma.sync m8n8k4; one warp per 8 rows; f64 with
 *     n in {8, 16, 24, 32}), 5 = FP32 register blocks (one thread per 4x4
 *     block of X A, X transposed in shared memory; f32, n >= 8, n padded to
 *     a multiple of 4 with zeros), 6 = two rows of X per thread (rows h and
 *     h + ceil(n / 2); f32), 7 = bf16 on the tcgen05 tensor cores (bf16,
 *     16 <= n <= 64, one instance per block at a time: {7, 1}; accumulator in
 *     tensor memory, fp32 state in registers; a persistent grid whose blocks
 *     keep their tensor memory; bounded waits counted like the LTimes tensor-
 *     core kernels', see cj_handle_wait_timeouts), 8 = FP32 register blocks
 *     of 4 rows x 8 columns (as 5 with columns padded to a multiple of 8:
 *     three 16-byte shared-memory reads per 32 fused multiply-adds).
 *     Default: n <= 4 -> {2, 128}; f32 grouped with n >= 17 -> {5, 1};
 *     f32 with n >= 32 -> {8, max(1, round(128 / t))}, t = ceil(n / 4) *
 *     ceil(n / 8) threads per instance; f32 with n >= 9 ->
 *     {6, max(1, 128 / ceil(n / 2))}; otherwise n <= 32 ->
 *     {1, max(1, 256 / n)};
 *     else {1, max(1, 128 / n)}; bf16 -> {3, max(1, 128 / n16)} with n16 = n
 *     rounded up to a multiple of 16 (mapping 3: one warp per 16 rows,
 *     bf16 operands, fp32 accumulate and state).
 *   mass operator: {elements per block, form, 0, 0}; form 0: an element owns
 *     max(D, Q)^2 threads and two shared-memory buffers of max(D, Q)^d values;
 *     form 1: the same on a persistent grid whose blocks stage the next
 *     group's x and op with cp.async while computing the current one (two
 *     stages of x and op in shared memory besides); form 2 (2-D with
 *     D Q + D^2 <= 80): one thread per element, every stage in registers.
 *     Default: form 2 with 128 elements where it applies, else form 0 with
 *     max(1, 256 / max(D, Q)^2) elements, fewer if the buffers of a block
 *     would exceed 96 KiB.
 *   Eigen recurrence: {mapping, instances per block, 0, 0}; M_k of every
 *     instance in shared memory, two buffers; mapping 1 = one thread per row
 *     of M, 2 = two rows per thread (rows h and h + ceil(n / 2); f32 only;
 *     same results bit for bit).  Default: f32 with n >= 2 -> mapping 2,
 *     else 1; instances per block max(1, 128 / t) with t = ceil(n / 2) or n
 *     threads per instance, fewer if both buffers would exceed 96 KiB.
 *   LTimes: {TG, TZ, threads, (PIPE << 20) | (MODE << 16) | (R << 8) | S}: a
 *     block covers TG x TZ (g, z) columns at a time (a persistent grid).
 *     MODE 0: the box with all d is staged in shared memory and each thread
 *     accumulates R columns x S moments on the FMA pipe (the last moment
 *     group may be partial), threads = (TG * TZ / R) * ceil(m / S).
 *     MODE 1 (f64, S = 8, d a multiple of 4): FP64 tensor cores (mma.sync
 *     m8n8k4), each warp 8R columns x all moments, threads =
 *     32 * TG * TZ / (8 R).
 *     MODE 2 (f32, R = 1, S = 8, d a multiple of 8): 3xTF32 on mma.sync
 *     m16n8k8, threads = 32 * TG * TZ / 16.
 *     PIPE 1 (modes 0-2): two tile buffers, the next tile loaded with cp.async
 *     while the current one is contracted.
 *     MODE 3 (f32, no PIPE, R <= 4): columns read straight from global memory,
 *     S moments per thread (S = 0: all, else a multiple of 4 below m),
 *     threads = TG * TZ / R * ceil(m / S).
 *     MODE 4 (f32, TG * TZ = 128, m <= 128 after the LPlusTimes swap): 3xTF32
 *     on tcgen05.mma kind::tf32 with the accumulator in tensor memory; R =
 *     operand stages (2..8), S = producer warps (2, 4 or 8), threads =
 *     32 * (5 + S), PIPE = the producers' register prefetch depth (0 auto).
 *     MODE 5: as mode 4 with `in` brought in by TMA (PIPE = boxes in flight,
 *     2..8; S = converter warps, threads = 32 * (6 + S); the box extent of
 *     in's innermost axis must be a multiple of 4).  A launch whose `in`
 *     admits no TMA tensor map (innermost extent not a multiple of 4, or not
 *     16-byte aligned) runs the mode-4 kernel of the same tile instead
 *     (cj_stats counts both).
 *     MODE 6: as mode 5 with the tf32 operand of `in` in tensor memory
 *     instead of shared memory (the converters write it with tcgen05.st and
 *     the MMAs read it from there): R = TMEM operand stages of 64 columns
 *     (2 <= R, 2 * ceil32(ceil16(m)) + 64 R <= 512), S = converter warps (4
 *     or 8), threads = 32 * (6 + S), PIPE = boxes in flight (2..8).  Its
 *     fallback without a tensor map is the mode-4 kernel with R 2, S 8.
 *     Default: call orders 1 and 4 "g-fast" (g is the fastest axis) and 0
 *     and 2 "z-fast"; TG = 1 if neither in nor out is g-fast, 8 if one is
 *     g-fast and the other z-fast, 32 otherwise.  f32 with m <= 128: TZ =
 *     128 / TG, MODE 6 with R 4, S 4 (320 threads) and the largest PIPE in
 *     {6, ..., 2} that fits 220 KiB of shared memory (and the mode-4
 *     fallback fits too), else MODE 5 with R 2, S 8 (448 threads) and the
 *     largest PIPE in {4, 3, 2} that fits, else MODE 4 with R 2, S 8
 *     (416 threads) if that fits.  Otherwise CT = 64 columns, TZ = CT / TG;
 *     f64: R 1, S 9, threads 64 * ceil(m / 9) (m = 36: 256); f32: PIPE 1,
 *     R 2, S 12, threads 32 * ceil(m / 12).  The FP64 tensor-core mappings
 *     are autotuner candidates, not defaults: on B300 mma.sync f64 issues on
 *     the FP64 pipe and is not faster than DFMA.
 */
typedef struct {
    int32_t dtype, n, layout_a, layout_b, m, d;
    int32_t tile[4];
    uint32_t flags;
} cj_template_args;

/* An instantiation.  Owned by the library, valid until cj_shutdown. */
typedef struct cj_handle_s *cj_handle;

typedef struct {
    uint64_t requests, cache_hits, compiles_ok, compiles_failed, aot_hits;
    uint64_t launches_generic, launches_aot, launches_jit;
    double compile_ms_p50, compile_ms_p95, lookup_ns_p50;
    /* LTimes tile modes 5 and 6: launches fed by TMA, and launches that fell back to
     * the mode-4 kernel because `in` admitted no tensor map (innermost extent
     * not a multiple of 4 floats, or `in` not 16-byte aligned) */
    uint64_t launches_tma, launches_tma_fallback;
    /* grouped plans: launches of a plan's dispatcher issued from the host
     * (cj_group_plan_launch without CJ_PLAN_GRAPH, or a graph capture) */
    uint64_t launches_dispatch;
    /* Expired bounded waits of the tensor-core LTimes kernels (tile modes
     * 4-6), summed over every run-time-compiled module and not yet cleared
     * through cj_handle_wait_timeouts(reset != 0).  A block whose wait expired
     * stopped early: any output written by a launch before a non-zero count
     * was seen is incomplete and must not be used.  Reading it synchronizes
     * the device when such a module is loaded (cj_stats then waits for all
     * queued work); it is 0 without synchronizing otherwise. */
    uint64_t wait_timeouts;
} cj_stats_t;

/* Initialise the library for `device` (idempotent for the same device).
 * Checks that the device is compute capability 10.3, loads the generic and
 * AoT kernels, and warms NVRTC so that later compiles touch no file.
 * cfg may be NULL (async, 1 thread, AoT set on, cost model off). */
cj_status cj_init(const cj_config *cfg, int device);

/* Look up or create the instantiation of kernel k for the runtime template
 * arguments a; *out receives its handle.  Cache hit: no compile.  Miss: the
 * handle is created, serves launches with the generic kernel at once, and an
 * NVRTC compile is queued (sync mode: performed before returning).  Returns
 * CJ_ERR_INVALID_ARG for out-of-range arguments (n <= 0 or n > 64, layout out
 * of range, bf16 with n < 16, null pointers), CJ_ERR_COMPILE in sync mode if
 * compilation failed (the handle is still valid and runs the generic kernel). */
cj_status cj_specialize(cj_kernel_id k, const cj_template_args *a, cj_handle *out);

/* Wait up to timeout_ms (negative: forever) for h's compile.  CJ_OK: the
 * specialized kernel is in use.  CJ_ERR_TIMEOUT: still compiling.
 * CJ_ERR_COMPILE: compilation failed; launches keep using the generic kernel. */
cj_status cj_specialize_wait(cj_handle h, int timeout_ms);

/*
 * Launch h on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * args follows cuLaunchKernel's kernelParams convention: args[i] points at
 * the i-th argument value.
 *   UPDATE_CHAIN: {const T** A, T** X, const int32_t* T_steps}; A and X are
 *     batch * n * n elements, instance b at offset b * n * n, each stored in
 *     layout_a order; T_steps >= 1; batch >= 0 instances.
 *   LTIMES: {const T** L, const T** in, T** out, const int64_t* G,
 *     const int64_t* Z}; L is [m][d] row-major, in is d*G*Z elements in
 *     order layout_a, out is m*G*Z in order layout_b; batch is ignored.
 *   LPLUSTIMES: {const T** Lp, const T** out, T** in, const int64_t* G,
 *     const int64_t* Z}; Lp is [d][m] row-major, out is m*G*Z elements in
 *     order layout_b (read), in is d*G*Z elements in order layout_a
 *     (accumulated into).
 *   MASS: {const T** B1, const T** op, const T** x, T** y}; B1 is the 1-D
 *     basis at the quadrature points, [Q][D] row-major; op is batch * Q^d
 *     values (quadrature data per element), x and y batch * D^d (dofs per
 *     element), each element's values with the first index fastest; batch =
 *     elements.
 *   EIGEN_RECURRENCE: {const T** M0, T** M, const int32_t* repeat, const
 *     double* c}; M0 and M are batch*n*n elements (row-major instances); repeat
 *     >= 0 steps (0 copies M0 to M).
 *   UPDATE_CHAIN_GROUPED: {const int64_t** worklist, const T** A_pool,
 *     T** X_pool, int32_t** counter}; batch = work items.  Item i is three
 *     int64 {element offset of A_i and X_i in the pools, T_i, reserved}; items
 *     should be sorted by T descending.  counter is one int32 in device memory
 *     that must be 0 at launch (the kernel increments it once per chunk of
 *     items it hands out and once more per block).
 * T is double for CJ_F64, float for CJ_F32 and CJ_BF16 (fp32 state).
 * LTimes / LPlusTimes tiles of modes 3-6 (the f32 defaults) move in and out
 * in 16-byte vectors: both must be 16-byte aligned.
 * Never blocks on compilation.  Returns CJ_ERR_INVALID_ARG without launching
 * for null args, negative batch or misaligned mode 3-6 tensors; CJ_ERR_CUDA if
 * the launch failed. */
cj_status cj_launch(cj_handle h, void *const *args, int64_t batch, void *cuda_stream);

/* Counters since cj_init; compile times are NVRTC + module load wall time.
 * CJ_ERR_CUDA if reading wait_timeouts failed (the other fields are set). */
cj_status cj_stats(cj_stats_t *out);

/* Canonical key (64 hex chars + NUL, needs cap >= 65) and the variant that
 * launches use right now: 0 generic, 1 AoT, 2 JIT. Either output may be NULL. */
cj_status cj_handle_info(cj_handle h, char *key_hex, size_t cap, int *variant);

/* Per-thread register count and static shared memory of the kernel that h
 * launches now (cuFuncGetAttribute), for the register comparison of Sec. 5. */
cj_status cj_handle_regs(cj_handle h, int *regs_per_thread, int *static_smem);

/* Bounded waits that expired in h's run-time-compiled kernel since the
 * module was loaded (or last reset).  The tcgen05 LTimes kernels (tile modes
 * 4-6) wait on shared-memory barriers for at most about a second each; a block
 * whose wait expires stops, waits for its issued tensor-core work, frees its
 * tensor memory, adds one to this counter and returns, leaving its part of
 * `out` incomplete.  Synchronizes the device, then reads the counter of h's
 * own module; reset != 0 zeroes it afterwards.  *count = 0 for handles with
 * no such module (AoT, generic, or kernels without bounded waits).
 * CJ_ERR_INVALID_ARG: null h or count; CJ_ERR_NO_DEVICE: compile-only mode;
 * CJ_ERR_CUDA: the synchronize or the copy failed. */
cj_status cj_handle_wait_timeouts(cj_handle h, uint32_t *count, int reset);

/*
 * Grouped plan for an uneven batch (many instances of different N and T in
 * one launch; the lookup cost is paid once per distinct N, Sec. 5.1).
 * Instance k has size n[k] (1..64) and steps[k] (>= 1); its A and X occupy
 * n[k]^2 row-major elements of the pools, at the exclusive prefix sum of
 * n[j]^2 over j < k.  The plan groups instances by n, requests one
 * UPDATE_CHAIN_GROUPED instantiation per group (tile 0 = default), orders
 * each group's items by T descending, and keeps work lists and counters in
 * device memory it owns.  dtype: CJ_F64, CJ_F32 or CJ_BF16 (pools in fp32;
 * groups with n >= 16 on bf16 tensor cores, the others in fp32).  flags: 0, or
 * CJ_FLAG_GENERIC to run every group on the generic grouped kernel.
 * Dispatcher: unless CJ_FLAG_GENERIC, the plan also generates one kernel for
 * the whole batch -- a persistent loop whose blocks take tickets (one chunk
 * of one group each, ordered by cost T n^3, longest first) from a counter
 * and run the ticket's group body, every body instantiated for the same
 * block size -- and requests its compilation (in the background in async
 * mode).  Launches use it once it is compiled; until then, or if it fails
 * to compile, or with CJ_PLAN_PER_GROUP, they launch one kernel per group.
 */
typedef struct cj_group_plan_s *cj_group_plan;
cj_status cj_group_plan_create(int32_t dtype, int64_t count, const int32_t *n, const int32_t *steps,
                               uint32_t flags, cj_group_plan *out);
/* Launch the plan on `cuda_stream`.  use_graph is a set of CJ_PLAN_* flags.
 * With the dispatcher ready (and no CJ_PLAN_PER_GROUP): one counter reset and
 * one dispatcher launch on cuda_stream.  Otherwise every group's kernel:
 * groups run concurrently on forked streams joined back into cuda_stream.
 * CJ_PLAN_GRAPH: the first call captures the whole launch (counter reset
 * included) into a CUDA graph on a stream of the plan's own and launches it
 * on cuda_stream; later calls replay it (re-captured when the pools, the
 * form or a group's instantiation changed, e.g. from generic to JIT, or the
 * dispatcher became ready).  Without it: the launches are issued from the
 * calling thread (per group: on the plan's streams, up to 64).  The GPU
 * overlaps independent streams only as far as the CUDA context has
 * hardware work queues: CUDA_DEVICE_MAX_CONNECTIONS (default 8, at most
 * 32), which must be set in the environment before the context is created.
 * With 32, long FP64 plans ran faster with use_graph = 0 than as a graph,
 * whose overlap did not change with the setting; time both for a given
 * plan.  A plan owns one set of work counters: launches of the same plan are
 * ordered by cuda_stream, so two launches on streams the caller does not
 * order against each other race (use one plan per concurrent stream).  Pools
 * are caller-owned device memory. */
#define CJ_PLAN_GRAPH 0x1      /* cj_group_plan_launch: capture once, replay a CUDA graph */
#define CJ_PLAN_PER_GROUP 0x2  /* cj_group_plan_launch: one kernel per group even when the dispatcher is ready */
cj_status cj_group_plan_launch(cj_group_plan p, const void *A_pool, void *X_pool, void *cuda_stream,
                               int use_graph);
/* The plan's dispatcher: *state 0 none (a CJ_FLAG_GENERIC plan), 1 compiling,
 * 2 ready (launches use it), 3 failed to compile, 4 ready but not used (the
 * plan's autotuner timed one kernel per group faster); *n_tickets its work
 * tickets; *threads its block size; *blocks_per_sm the resident blocks per SM
 * of the variant in use (0 until it is compiled).  Any output may be NULL. */
cj_status cj_group_plan_dispatcher(cj_group_plan p, int32_t *state, int32_t *n_tickets, int32_t *threads,
                                   int32_t *blocks_per_sm);
/* Pin the plan's dispatcher to variant `variant` (0 .. *variants - 1; the
 * variants differ in the register cap of the launch bounds, for f32 in the
 * tile rule of the n >= 16 groups (rule 0 = 4 x 4 register blocks, mapping
 * 5; rule 1 = 4 x 8, mapping 8), and for bf16 in the block size (256 or 128
 * threads)).  Compiles it if needed (waits),
 * and makes later launches (and graph captures) use it, as the plan's
 * autotuner does with the fastest.  variant < 0 only reports *variants (may
 * be NULL; 0 for a plan without a dispatcher).  Not to be called while
 * another thread launches or destroys the same plan.  CJ_ERR_INVALID_ARG:
 * null plan, no dispatcher or variant out of range; CJ_ERR_COMPILE: it failed
 * to compile; CJ_ERR_NO_DEVICE in compile-only mode. */
cj_status cj_group_plan_use_dispatcher(cj_group_plan p, int32_t variant, int32_t *variants);
/* Wait up to timeout_ms (negative: forever) for the instantiations of every
 * group of p to finish compiling.  CJ_OK: every group launches its
 * specialized kernel.  CJ_ERR_TIMEOUT: some are still compiling (launches
 * meanwhile use the generic grouped kernel for them).  CJ_ERR_COMPILE: a
 * group's compilation failed; that group keeps the generic kernel. */
cj_status cj_group_plan_wait(cj_group_plan p, int timeout_ms);
/* Groups in the plan and pool elements it expects. */
/* Autotune a plan's tiles (the batching pattern's autotuned tiles): for each
 * of the max_groups most expensive groups (0: all), every candidate tile of
 * the grouped kernel (cj_candidates, at most 256 instances per chunk) is
 * compiled and timed on the group's own work list on `stream` (median of reps
 * launches after one warm-up, CUDA events); the fastest replaces the group's
 * tile, and the next graph launch re-captures.  Then, once the plan's
 * dispatcher is compiled (this waits for it), the whole launch is timed in
 * both forms -- every dispatcher variant (cj_group_plan_use_dispatcher), and
 * one kernel per group; each as a graph and issued directly, the mean of
 * max(reps, 10) launches issued back to back after a warm-up -- and later
 * launches use the fastest.  X_pool is written: every timed
 * launch computes its group's instances.  *changed (may be NULL) receives the
 * number of groups whose tile changed.  Synchronous; compiles run on the
 * background threads in async mode.  Not to be called while another thread
 * launches or destroys the same plan.  CJ_ERR_INVALID_ARG: null plan or pools;
 * CJ_ERR_NO_DEVICE in compile-only mode; CJ_ERR_CUDA if a launch or timing
 * call failed. */
cj_status cj_group_plan_autotune(cj_group_plan p, const void *A_pool, void *X_pool, void *cuda_stream,
                                 int32_t max_groups, int32_t reps, int32_t *changed);
cj_status cj_group_plan_info(cj_group_plan p, int32_t *n_groups, int64_t *pool_elems);
cj_status cj_group_plan_destroy(cj_group_plan p);

/* Measured throughput of this GPU in TFLOP/s (2 flops per multiply-add) for
 * dtype CJ_F64 or CJ_F32: tensor = 0, independent fused multiply-add chains
 * over every SM; tensor = 1 (f64 only), independent mma.sync m8n8k4 FP64
 * tensor-core chains.  Timed with CUDA events on cuda_stream.  The roofline
 * denominators of the arithmetic-bound kernels. */
cj_status cj_measure_fma_peak(int32_t dtype, int32_t tensor, void *cuda_stream, double *tflops);

/*
 * Allocation-free uneven update chain.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory --
 * code running under a device-memory budget owned by another allocator (a
 * framework's caching allocator, an arena in an embedded or real-time
 * deployment) and code on latency-critical paths, where cudaMalloc/cudaFree
 * may synchronize the device.  It computes what cj_group_plan_create +
 * cj_group_plan_launch compute for the same instances (same pool layout:
 * instance k at the exclusive prefix sum of n[j]^2, row-major), using the
 * generic runtime-N kernel per group, groups one after another on
 * cuda_stream.  It calls no cudaMalloc/cudaFree and no allocating library
 * routine, and does not need cj_init.
 *   Scratch: the work list and per-n counters live in one fixed file-scope
 *   __device__ array of CJ_NOALLOC_MAX_INSTANCES * 24 + 256 bytes (about
 *   1.5 MiB) that every GPU which loads this library holds until the process
 *   exits.  count > CJ_NOALLOC_MAX_INSTANCES returns CJ_ERR_INVALID_ARG.
 *   The first call on a device looks up that array's device address (with
 *   the device current) and sets kernel attributes.  cj_shutdown forgets
 *   this set-up; a caller that resets a device (cudaDeviceReset) calls
 *   cj_shutdown before the next call on it.
 *   Every call reuses the same array and resets its counters at the start;
 *   calls whose work overlaps on the GPU (other streams, or other host
 *   threads on the same device) race on it and must be serialized by the
 *   caller.  The work list is built in pageable host memory that the call
 *   owns and copied with cudaMemcpyAsync on cuda_stream: the CUDA runtime
 *   stages such a copy, so the call returns only after the work queued
 *   earlier on cuda_stream has finished, and the call must not be made while
 *   cuda_stream (or its device, in global capture mode) is being captured
 *   into a CUDA graph.
 * dtype: CJ_F64 or CJ_F32; n[k] in 1..64; steps[k] >= 1; A_pool, X_pool are
 * caller-owned device memory.  Errors: CJ_ERR_INVALID_ARG (bad arguments,
 * too many instances), CJ_ERR_NO_DEVICE, CJ_ERR_CUDA (cj_last_error has the
 * reason). */
#define CJ_NOALLOC_MAX_INSTANCES 65536
cj_status cj_update_chain_uneven_noalloc(int32_t dtype, int64_t count, const int32_t *n, const int32_t *steps,
                                         const void *A_pool, void *X_pool, void *cuda_stream);

/*
 * Autotuner and learned cost model (the paper's future work: profiling
 * information used to guide autotuning of JIT-compiled code, Sec. 6).
 *
 * cj_candidates: the tile space searched for a request (tile fields ignored);
 *   writes min(cap, count) tiles as int32[4] rows.
 * cj_autotune: compiles every candidate (JIT) and times it on the caller's
 *   device buffers (launch_args/batch as for cj_launch, each candidate
 *   warmed once, then the median of reps launches, CUDA events on
 *   cuda_stream).  best_tile gets the fastest; times_ms[i] (cap entries)
 *   the time of candidate i in cj_candidates order (INFINITY if it did not
 *   compile).
 * cj_featurize: the CJ_FEATURES-float input vector of the cost model for
 *   (request, tile) at `batch` instances (chain) or columns G*Z (LTimes)
 *   and `steps` (chain T); the last feature is 1 for the tile the default
 *   rule picks for the request, else 0.  Not defined for CJ_K_MASS (whose
 *   tiles are autotuned exhaustively): CJ_ERR_INVALID_ARG.
 * cj_mlp_*: an in_features -> 64 -> 64 -> 1 ReLU network in FP32 on the
 *   device (library-owned).  Parameters are one flat vector in the order
 *   W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3.  forward: y = f(X)
 *   for X[B][F] (device pointers).  grad: gradient of the mean squared
 *   error (1/B) sum (y - t)^2 into grad (device, count floats) and the loss
 *   into *loss (device, may be NULL), parameters unchanged.  train_step: the
 *   same gradient, then one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 *   rate lr).  Deterministic: no atomics.  create draws weights from
 *   SplitMix64(seed), U(-s, s) with s = sqrt(3 / fan_in), biases 0.
 * cj_cost_model_use: install m (in_features == CJ_FEATURES) for
 *   cj_specialize requests with tile = {0,0,0,0} when cj_config.use_cost_model
 *   is set (NULL uninstalls); the decision is cached per request.  Only
 *   UPDATE_CHAIN and LTIMES requests consult it; the other kernels keep
 *   their default rule.  cj_cost_model_use_ensemble installs count networks
 *   whose predictions are averaged (count 0 uninstalls); the library keeps
 *   the pointers, not copies: destroying an installed network uninstalls the
 *   ensemble.
 * cj_choose_tile: the candidate with the lowest predicted log time (the
 *   mean over the installed networks; each network's output is read as the
 *   natural log of the time), for any kernel with candidates (a model
 *   trained on other kernels extrapolates), except that the default rule's
 *   tile is kept unless another candidate is predicted faster by more than
 *   log(1.10).  The cost-model hook of cj_specialize decides the same way.
 */
#define CJ_FEATURES 32
typedef struct cj_mlp_s *cj_mlp;
cj_status cj_candidates(cj_kernel_id k, const cj_template_args *a, int32_t *tiles, int32_t cap, int32_t *count);
cj_status cj_autotune(cj_kernel_id k, const cj_template_args *a, void *const *launch_args, int64_t batch,
                      void *cuda_stream, int32_t reps, int32_t best_tile[4], float *times_ms, int32_t cap,
                      int32_t *count);
cj_status cj_featurize(cj_kernel_id k, const cj_template_args *a, int64_t batch, int32_t steps,
                       const int32_t tile[4], float *out);
cj_status cj_mlp_create(int32_t in_features, uint64_t seed, cj_mlp *out);
cj_status cj_mlp_set_params(cj_mlp m, const float *host, int64_t count);
cj_status cj_mlp_get_params(cj_mlp m, float *host, int64_t cap, int64_t *count);
cj_status cj_mlp_forward(cj_mlp m, const float *X, int64_t B, float *y, void *cuda_stream);
cj_status cj_mlp_grad(cj_mlp m, const float *X, const float *t, int64_t B, float *grad, float *loss,
                      void *cuda_stream);
cj_status cj_mlp_train_step(cj_mlp m, const float *X, const float *t, int64_t B, float lr, float *loss,
                            void *cuda_stream);
cj_status cj_mlp_destroy(cj_mlp m);
cj_status cj_cost_model_use(cj_mlp m);
cj_status cj_cost_model_use_ensemble(const cj_mlp *m, int32_t count);
cj_status cj_choose_tile(cj_kernel_id k, const cj_template_args *a, int64_t batch, int32_t steps,
                         int32_t tile_out[4], float *predicted_log_time);

/* Thread-local description of the last error on this thread ("" if none). */
const char *cj_last_error(void);

/* Wait for queued compiles, unload modules, free every handle and plan. */
cj_status cj_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* CJ_H */
