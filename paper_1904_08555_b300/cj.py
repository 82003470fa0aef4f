"""ctypes binding of libcj (include/cj.h): argument marshalling only.

Every step of the path runs in libcj's kernels.  If the shared library is
missing it is built from source (nvcc / g++); if that fails the import fails:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

CJ_OK, CJ_ERR_INVALID_ARG, CJ_ERR_NOT_INITIALIZED, CJ_ERR_NO_DEVICE = 0, 1, 2, 3
CJ_ERR_UNSUPPORTED_ARCH, CJ_ERR_COMPILE, CJ_ERR_CUDA, CJ_ERR_OOM = 4, 5, 6, 7
CJ_ERR_TIMEOUT, CJ_ERR_PENDING = 8, 9

K_UPDATE_CHAIN, K_LTIMES, K_UPDATE_CHAIN_GROUPED, K_LPLUSTIMES, K_EIGEN_RECURRENCE, K_MASS = 1, 2, 3, 4, 5, 6
F64, F32, BF16 = 0, 1, 2
FLAG_GENERIC, FLAG_NO_AOT, FLAG_INJECT_COMPILE_ERROR, FLAG_INJECT_WAIT_TIMEOUT = 0x1, 0x2, 0x100, 0x200
CFG_COMPILE_ONLY = 0x1
PLAN_GRAPH, PLAN_PER_GROUP = 0x1, 0x2
VARIANT_NAMES = ("generic", "aot", "jit")

EXPORTS = ("cj_init", "cj_specialize", "cj_specialize_wait", "cj_launch", "cj_stats", "cj_handle_info",
           "cj_handle_regs", "cj_handle_wait_timeouts", "cj_group_plan_create", "cj_group_plan_launch",
           "cj_group_plan_autotune", "cj_group_plan_wait", "cj_group_plan_dispatcher", "cj_group_plan_use_dispatcher",
           "cj_group_plan_info",
           "cj_group_plan_destroy", "cj_measure_fma_peak", "cj_update_chain_uneven_noalloc", "cj_candidates",
           "cj_autotune", "cj_featurize", "cj_mlp_create", "cj_mlp_set_params", "cj_mlp_get_params",
           "cj_mlp_forward", "cj_mlp_grad", "cj_mlp_train_step", "cj_mlp_destroy", "cj_cost_model_use", "cj_cost_model_use_ensemble",
           "cj_choose_tile", "cj_last_error", "cj_shutdown")
FEATURES = 32


class CJError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("sync", ctypes.c_uint32), ("compile_threads", ctypes.c_uint32),
                ("use_cost_model", ctypes.c_uint32), ("enable_aot_set", ctypes.c_uint32),
                ("debug_bounds", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class TemplateArgs(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("n", ctypes.c_int32), ("layout_a", ctypes.c_int32),
                ("layout_b", ctypes.c_int32), ("m", ctypes.c_int32), ("d", ctypes.c_int32),
                ("tile", ctypes.c_int32 * 4), ("flags", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests", "cache_hits", "compiles_ok", "compiles_failed",
                                               "aot_hits", "launches_generic", "launches_aot", "launches_jit")] + \
               [(n, ctypes.c_double) for n in ("compile_ms_p50", "compile_ms_p95", "lookup_ns_p50")] + \
               [(n, ctypes.c_uint64) for n in ("launches_tma", "launches_tma_fallback", "launches_dispatch",
                                               "wait_timeouts")]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libcj.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.cj_init.argtypes = [ctypes.POINTER(Config), ctypes.c_int]
        L.cj_specialize.argtypes = [ctypes.c_int, ctypes.POINTER(TemplateArgs), ctypes.POINTER(P)]
        L.cj_specialize_wait.argtypes = [P, ctypes.c_int]
        L.cj_launch.argtypes = [P, ctypes.POINTER(P), i64, P]
        L.cj_stats.argtypes = [ctypes.POINTER(Stats)]
        L.cj_handle_info.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]
        L.cj_handle_regs.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.cj_handle_wait_timeouts.argtypes = [P, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        L.cj_group_plan_create.argtypes = [i32, i64, P, P, ctypes.c_uint32, ctypes.POINTER(P)]
        L.cj_group_plan_launch.argtypes = [P, P, P, P, ctypes.c_int]
        L.cj_group_plan_autotune.argtypes = [P, P, P, P, i32, i32, ctypes.POINTER(i32)]
        L.cj_group_plan_wait.argtypes = [P, ctypes.c_int]
        L.cj_group_plan_dispatcher.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                               ctypes.POINTER(i32)]
        L.cj_group_plan_use_dispatcher.argtypes = [P, i32, ctypes.POINTER(i32)]
        L.cj_group_plan_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.cj_group_plan_destroy.argtypes = [P]
        L.cj_measure_fma_peak.argtypes = [i32, i32, P, ctypes.POINTER(ctypes.c_double)]
        L.cj_update_chain_uneven_noalloc.argtypes = [i32, i64, P, P, P, P, P]
        TA = ctypes.POINTER(TemplateArgs)
        L.cj_candidates.argtypes = [ctypes.c_int, TA, P, i32, ctypes.POINTER(i32)]
        L.cj_autotune.argtypes = [ctypes.c_int, TA, ctypes.POINTER(P), i64, P, i32, P, P, i32, ctypes.POINTER(i32)]
        L.cj_featurize.argtypes = [ctypes.c_int, TA, i64, i32, P, P]
        L.cj_mlp_create.argtypes = [i32, ctypes.c_uint64, ctypes.POINTER(P)]
        L.cj_mlp_set_params.argtypes = [P, P, i64]
        L.cj_mlp_get_params.argtypes = [P, P, i64, ctypes.POINTER(i64)]
        L.cj_mlp_forward.argtypes = [P, P, i64, P, P]
        L.cj_mlp_grad.argtypes = [P, P, P, i64, P, P, P]
        L.cj_mlp_train_step.argtypes = [P, P, P, i64, ctypes.c_float, P, P]
        L.cj_mlp_destroy.argtypes = [P]
        L.cj_cost_model_use.argtypes = [P]
        L.cj_cost_model_use_ensemble.argtypes = [ctypes.POINTER(P), i32]
        L.cj_choose_tile.argtypes = [ctypes.c_int, TA, i64, i32, P, ctypes.POINTER(ctypes.c_float)]
        L.cj_last_error.restype = ctypes.c_char_p
        L.cj_shutdown.argtypes = []
        for name in EXPORTS:
            if name != "cj_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def last_error() -> str:
    return load().cj_last_error().decode(errors="replace")


def _check(rc: int, where: str, ok=(CJ_OK,)):
    if rc not in ok:
        raise CJError(rc, where, last_error())
    return rc


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream, *tensors) -> int:
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for t in tensors:
        if hasattr(t, "is_cuda") and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return 0


def init(sync=False, compile_threads=1, use_cost_model=False, enable_aot_set=True,
         compile_only=False, device=0) -> None:
    cfg = Config(int(sync), compile_threads, int(use_cost_model), int(enable_aot_set), 0,
                 CFG_COMPILE_ONLY if compile_only else 0)
    _check(load().cj_init(ctypes.byref(cfg), device), "cj_init")


def shutdown() -> None:
    _check(load().cj_shutdown(), "cj_shutdown")


class Handle:
    """An instantiation returned by cj_specialize (owned by the library)."""

    def __init__(self, ptr: int, kernel: int, args: TemplateArgs):
        self.ptr = ptr
        self.kernel = kernel
        self.dtype = args.dtype
        self.n = args.n
        self.m, self.d = args.m, args.d

    def info(self):
        buf = ctypes.create_string_buffer(65)
        var = ctypes.c_int(-1)
        _check(load().cj_handle_info(self.ptr, buf, 65, ctypes.byref(var)), "cj_handle_info")
        return buf.value.decode(), var.value

    @property
    def key_hex(self) -> str:
        return self.info()[0]

    @property
    def variant(self) -> str:
        return VARIANT_NAMES[self.info()[1]]

    def regs(self):
        r, s = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().cj_handle_regs(self.ptr, ctypes.byref(r), ctypes.byref(s)), "cj_handle_regs")
        return r.value, s.value

    def wait_timeouts(self, reset: bool = False) -> int:
        """Expired bounded waits in this handle's JIT module (synchronizes the device)."""
        c = ctypes.c_uint32(0)
        _check(load().cj_handle_wait_timeouts(self.ptr, ctypes.byref(c), int(reset)), "cj_handle_wait_timeouts")
        return c.value

    def wait(self, timeout_ms: int = -1) -> int:
        return load().cj_specialize_wait(self.ptr, timeout_ms)

    def __eq__(self, other):
        return isinstance(other, Handle) and other.ptr == self.ptr

    def __hash__(self):
        return hash(self.ptr)


def specialize(kernel: int, dtype: int, n=0, layout_a=0, layout_b=0, m=0, d=0, tile=(0, 0, 0, 0),
               flags=0, allow_compile_error=False) -> Handle:
    a = TemplateArgs(dtype, n, layout_a, layout_b, m, d, (ctypes.c_int32 * 4)(*tile), flags)
    out = ctypes.c_void_p()
    ok = (CJ_OK, CJ_ERR_COMPILE) if allow_compile_error else (CJ_OK,)
    _check(load().cj_specialize(kernel, ctypes.byref(a), ctypes.byref(out)), "cj_specialize", ok)
    return Handle(out.value, kernel, a)


def _launch(h: Handle, vals, batch: int, stream: int) -> None:
    arr = (ctypes.c_void_p * len(vals))(*[ctypes.cast(ctypes.pointer(v), ctypes.c_void_p) for v in vals])
    _check(load().cj_launch(h.ptr, arr, batch, stream), "cj_launch")


def _check_sizes(h: Handle, where: str, batch: int, *pairs) -> None:
    """Each (tensor, elements) pair: a contiguous CUDA tensor of the handle's
    element type holding at least that many elements (skipped for raw device
    addresses and for an empty batch, which reads and writes nothing)."""
    if batch > 0:
        for t, elems in pairs:
            _check_pool(t, h.dtype, elems, where)


def launch_update_chain(h: Handle, A, X, steps: int, batch: int | None = None, stream=None) -> None:
    """X_T for every instance: A, X hold batch*n*n elements (tensors or device pointers)."""
    if batch is None:
        batch = A.numel() // (h.n * h.n)
    _check_sizes(h, "cj_launch", batch, (A, batch * h.n * h.n), (X, batch * h.n * h.n))
    vals = [ctypes.c_void_p(_ptr(A)), ctypes.c_void_p(_ptr(X)), ctypes.c_int32(steps)]
    _launch(h, vals, batch, _stream(stream, A, X))


def launch_ltimes(h: Handle, L, x, out, G: int, Z: int, stream=None) -> None:
    """out = L . in: L [m][d], x (d*G*Z, layout_a), out (m*G*Z, layout_b)."""
    _check_sizes(h, "cj_launch", G * Z, (L, h.m * h.d), (x, h.d * G * Z), (out, h.m * G * Z))
    vals = [ctypes.c_void_p(_ptr(L)), ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out)),
            ctypes.c_int64(G), ctypes.c_int64(Z)]
    _launch(h, vals, Z, _stream(stream, L, x, out))


def launch_lplustimes(h: Handle, Lp, out, x, G: int, Z: int, stream=None) -> None:
    """x += Lp . out (LPlusTimes): Lp [d][m], out (m*G*Z, layout_b), x (d*G*Z, layout_a)."""
    _check_sizes(h, "cj_launch", G * Z, (Lp, h.m * h.d), (out, h.m * G * Z), (x, h.d * G * Z))
    vals = [ctypes.c_void_p(_ptr(Lp)), ctypes.c_void_p(_ptr(out)), ctypes.c_void_p(_ptr(x)),
            ctypes.c_int64(G), ctypes.c_int64(Z)]
    _launch(h, vals, Z, _stream(stream, Lp, out, x))


def launch_eigen(h: Handle, M0, M, repeat: int, c: float = 5e-5, batch=None, stream=None) -> None:
    """M_{k+1} = Ones + c (M_k + M_k M_k), repeat times, from M0 (batch*n*n, row-major) into M."""
    if batch is None:
        batch = M0.numel() // (h.n * h.n) if hasattr(M0, "numel") else 0
    _check_sizes(h, "cj_launch", batch, (M0, batch * h.n * h.n), (M, batch * h.n * h.n))
    vals = [ctypes.c_void_p(_ptr(M0)), ctypes.c_void_p(_ptr(M)), ctypes.c_int32(repeat), ctypes.c_double(c)]
    _launch(h, vals, batch, _stream(stream, M0, M))


def launch_mass(h: Handle, B1, op, x, y, ne: int, stream=None) -> None:
    """y_e = B^T diag(op_e) B x_e for ne elements (B1: [Q][D]; op: ne*Q^d; x, y: ne*D^d)."""
    D, Q, dim = h.n, h.m, h.d
    _check_sizes(h, "cj_launch", ne, (B1, Q * D), (op, ne * Q ** dim), (x, ne * D ** dim), (y, ne * D ** dim))
    vals = [ctypes.c_void_p(_ptr(B1)), ctypes.c_void_p(_ptr(op)), ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(y))]
    _launch(h, vals, ne, _stream(stream, B1, op, x, y))


def launch_grouped(h: Handle, items, A_pool, X_pool, counter, n_items: int, stream=None) -> None:
    vals = [ctypes.c_void_p(_ptr(items)), ctypes.c_void_p(_ptr(A_pool)), ctypes.c_void_p(_ptr(X_pool)),
            ctypes.c_void_p(_ptr(counter))]
    _launch(h, vals, n_items, _stream(stream, A_pool, X_pool))


def measure_fma_peak(dtype: int, stream=None, tensor: bool = False) -> float:
    """Measured throughput (TFLOP/s) for F64 or F32; tensor=True: FP64 mma.sync."""
    out = ctypes.c_double(0.0)
    _check(load().cj_measure_fma_peak(dtype, int(tensor), _stream(stream), ctypes.byref(out)),
           "cj_measure_fma_peak")
    return out.value


NOALLOC_MAX_INSTANCES = 65536


def _check_pool(t, dtype: int, elems: int, where: str) -> None:
    """A pool tensor must be a contiguous CUDA tensor of the dtype's element
    type (fp32 state for BF16) holding at least `elems` elements; otherwise
    the kernels would read or write past the caller's memory.  Raw integer
    device addresses are passed through unchecked."""
    if t is None or isinstance(t, int):
        return
    import torch
    want = torch.float64 if dtype == F64 else torch.float32
    if not t.is_cuda or t.dtype != want or not t.is_contiguous() or t.numel() < elems:
        raise CJError(CJ_ERR_INVALID_ARG, where,
                      f"pool must be a contiguous CUDA {want} tensor of at least {elems} elements "
                      f"(got {t.dtype}, {t.numel()} elements, device {t.device}, "
                      f"contiguous {t.is_contiguous()})")


def update_chain_uneven_noalloc(dtype: int, n, steps, A_pool, X_pool, stream=None) -> None:
    """cj_update_chain_uneven_noalloc: the uneven update chain without any
    device allocation (scratch in a fixed array inside the library); for
    callers that must not allocate device memory."""
    import numpy as np
    n = np.ascontiguousarray(n, dtype=np.int32)
    steps = np.ascontiguousarray(steps, dtype=np.int32)
    elems = int(np.sum(n.astype(np.int64) ** 2))
    _check_pool(A_pool, dtype, elems, "cj_update_chain_uneven_noalloc")
    _check_pool(X_pool, dtype, elems, "cj_update_chain_uneven_noalloc")
    _check(load().cj_update_chain_uneven_noalloc(dtype, len(n), n.ctypes.data, steps.ctypes.data, _ptr(A_pool),
                                                  _ptr(X_pool), _stream(stream, A_pool, X_pool)),
           "cj_update_chain_uneven_noalloc")


def stats() -> dict:
    s = Stats()
    _check(load().cj_stats(ctypes.byref(s)), "cj_stats")
    return {name: getattr(s, name) for name, _ in Stats._fields_}


class GroupPlan:
    """cj_group_plan_*: uneven batch grouped by n, launched as one (graph) launch."""

    def __init__(self, dtype: int, n, steps, flags: int = 0):
        import numpy as np
        n = np.ascontiguousarray(n, dtype=np.int32)
        steps = np.ascontiguousarray(steps, dtype=np.int32)
        out = ctypes.c_void_p()
        _check(load().cj_group_plan_create(dtype, len(n), n.ctypes.data, steps.ctypes.data, flags,
                                           ctypes.byref(out)), "cj_group_plan_create")
        self.ptr = out.value
        self.dtype = dtype
        g, e = ctypes.c_int32(0), ctypes.c_int64(0)
        _check(load().cj_group_plan_info(self.ptr, ctypes.byref(g), ctypes.byref(e)), "cj_group_plan_info")
        self.n_groups, self.pool_elems = g.value, e.value

    def launch(self, A_pool, X_pool, stream=None, use_graph=True, per_group=False) -> None:
        """One launch of the whole batch: the plan's dispatcher once it is
        compiled (unless per_group), else one kernel per group."""
        _check_pool(A_pool, self.dtype, self.pool_elems, "cj_group_plan_launch")
        _check_pool(X_pool, self.dtype, self.pool_elems, "cj_group_plan_launch")
        flags = (PLAN_GRAPH if use_graph else 0) | (PLAN_PER_GROUP if per_group else 0)
        _check(load().cj_group_plan_launch(self.ptr, _ptr(A_pool), _ptr(X_pool), _stream(stream, A_pool, X_pool),
                                           flags), "cj_group_plan_launch")

    def dispatcher(self) -> dict:
        """State of the plan's dispatcher: none, compiling, ready or failed."""
        st, nt, th, bp = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().cj_group_plan_dispatcher(self.ptr, ctypes.byref(st), ctypes.byref(nt), ctypes.byref(th),
                                               ctypes.byref(bp)), "cj_group_plan_dispatcher")
        return {"state": ("none", "compiling", "ready", "failed", "not used")[st.value], "tickets": nt.value,
                "threads": th.value, "blocks_per_sm": bp.value}

    def use_dispatcher(self, variant: int = -1) -> int:
        """Pin the dispatcher to `variant` (compiled if needed); returns the number of variants."""
        n = ctypes.c_int32(0)
        _check(load().cj_group_plan_use_dispatcher(self.ptr, variant, ctypes.byref(n)), "cj_group_plan_use_dispatcher")
        return n.value

    def autotune(self, A_pool, X_pool, stream=None, max_groups: int = 0, reps: int = 3) -> int:
        """Time every candidate tile per group (most expensive first) and keep the fastest; returns groups changed."""
        _check_pool(A_pool, self.dtype, self.pool_elems, "cj_group_plan_autotune")
        _check_pool(X_pool, self.dtype, self.pool_elems, "cj_group_plan_autotune")
        ch = ctypes.c_int32(0)
        _check(load().cj_group_plan_autotune(self.ptr, _ptr(A_pool), _ptr(X_pool), _stream(stream, A_pool, X_pool),
                                             max_groups, reps, ctypes.byref(ch)), "cj_group_plan_autotune")
        return ch.value

    def wait(self, timeout_ms: int = -1) -> None:
        """Block until every group's instantiation is compiled (async mode)."""
        _check(load().cj_group_plan_wait(self.ptr, timeout_ms), "cj_group_plan_wait")

    def destroy(self) -> None:
        if self.ptr:
            load().cj_group_plan_destroy(self.ptr)
            self.ptr = None


# ---------------------------------------------------------------------------
# autotuner and cost model
# ---------------------------------------------------------------------------
def _targs(dtype, n=0, layout_a=0, layout_b=0, m=0, d=0, tile=(0, 0, 0, 0), flags=0):
    return TemplateArgs(dtype, n, layout_a, layout_b, m, d, (ctypes.c_int32 * 4)(*tile), flags)


def candidates(kernel: int, dtype: int, n=0, layout_a=0, layout_b=0, m=0, d=0):
    """Candidate tiles (list of 4-tuples) searched for this request."""
    import numpy as np
    a = _targs(dtype, n, layout_a, layout_b, m, d)
    cnt = ctypes.c_int32(0)
    _check(load().cj_candidates(kernel, ctypes.byref(a), None, 0, ctypes.byref(cnt)), "cj_candidates")
    buf = np.zeros((cnt.value, 4), dtype=np.int32)
    _check(load().cj_candidates(kernel, ctypes.byref(a), buf.ctypes.data, cnt.value, ctypes.byref(cnt)),
           "cj_candidates")
    return [tuple(int(v) for v in row) for row in buf]


def featurize(kernel: int, dtype: int, batch: int, steps: int, tile, n=0, layout_a=0, layout_b=0, m=0, d=0):
    import numpy as np
    a = _targs(dtype, n, layout_a, layout_b, m, d)
    t = np.ascontiguousarray(tile, dtype=np.int32)
    out = np.zeros(FEATURES, dtype=np.float32)
    _check(load().cj_featurize(kernel, ctypes.byref(a), batch, steps, t.ctypes.data, out.ctypes.data),
           "cj_featurize")
    return out


def autotune(kernel: int, dtype: int, launch_vals, batch: int, stream, reps=3, n=0, layout_a=0, layout_b=0, m=0,
             d=0):
    """Exhaustive autotune on the caller's buffers; returns (best_tile, [(tile, ms), ...])."""
    import numpy as np
    a = _targs(dtype, n, layout_a, layout_b, m, d)
    cands = candidates(kernel, dtype, n, layout_a, layout_b, m, d)
    arr = (ctypes.c_void_p * len(launch_vals))(*[ctypes.cast(ctypes.pointer(v), ctypes.c_void_p) for v in launch_vals])
    best = np.zeros(4, dtype=np.int32)
    times = np.zeros(len(cands), dtype=np.float32)
    cnt = ctypes.c_int32(0)
    _check(load().cj_autotune(kernel, ctypes.byref(a), arr, batch, _stream(stream), reps, best.ctypes.data,
                              times.ctypes.data, len(cands), ctypes.byref(cnt)), "cj_autotune")
    return tuple(int(v) for v in best), list(zip(cands, [float(t) for t in times]))


def chain_launch_vals(A, X, steps):
    return [ctypes.c_void_p(_ptr(A)), ctypes.c_void_p(_ptr(X)), ctypes.c_int32(steps)]


def ltimes_launch_vals(L, x, out, G, Z):
    return [ctypes.c_void_p(_ptr(L)), ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(out)), ctypes.c_int64(G),
            ctypes.c_int64(Z)]


class MLP:
    """The cost model's F -> 64 -> 64 -> 1 ReLU network (device-resident, FP32)."""

    def __init__(self, in_features: int = FEATURES, seed: int = 0xC1A5):
        out = ctypes.c_void_p()
        _check(load().cj_mlp_create(in_features, seed, ctypes.byref(out)), "cj_mlp_create")
        self.ptr = out.value
        self.F = in_features
        self.P = 64 * in_features + 64 + 64 * 64 + 64 + 64 + 1

    def get_params(self):
        import numpy as np
        buf = np.zeros(self.P, dtype=np.float32)
        cnt = ctypes.c_int64(0)
        _check(load().cj_mlp_get_params(self.ptr, buf.ctypes.data, self.P, ctypes.byref(cnt)), "cj_mlp_get_params")
        return buf

    def set_params(self, v):
        import numpy as np
        v = np.ascontiguousarray(v, dtype=np.float32)
        _check(load().cj_mlp_set_params(self.ptr, v.ctypes.data, v.size), "cj_mlp_set_params")

    def forward(self, X, y, stream=None):
        _check(load().cj_mlp_forward(self.ptr, _ptr(X), X.shape[0], _ptr(y), _stream(stream, X, y)),
               "cj_mlp_forward")

    def grad(self, X, t, grad, loss=None, stream=None):
        _check(load().cj_mlp_grad(self.ptr, _ptr(X), _ptr(t), X.shape[0], _ptr(grad), _ptr(loss),
                                  _stream(stream, X, t)), "cj_mlp_grad")

    def train_step(self, X, t, lr, loss=None, stream=None):
        _check(load().cj_mlp_train_step(self.ptr, _ptr(X), _ptr(t), X.shape[0], lr, _ptr(loss),
                                        _stream(stream, X, t)), "cj_mlp_train_step")

    def use_as_cost_model(self):
        _check(load().cj_cost_model_use(self.ptr), "cj_cost_model_use")

    def destroy(self):
        if self.ptr:
            load().cj_mlp_destroy(self.ptr)
            self.ptr = None


def clear_cost_model():
    _check(load().cj_cost_model_use(None), "cj_cost_model_use")


def use_cost_model_ensemble(nets) -> None:
    """Install several networks; their predictions are averaged."""
    arr = (ctypes.c_void_p * len(nets))(*[n.ptr for n in nets])
    _check(load().cj_cost_model_use_ensemble(arr, len(nets)), "cj_cost_model_use_ensemble")


def choose_tile(kernel: int, dtype: int, batch: int, steps: int, n=0, layout_a=0, layout_b=0, m=0, d=0):
    import numpy as np
    a = _targs(dtype, n, layout_a, layout_b, m, d)
    out = np.zeros(4, dtype=np.int32)
    pred = ctypes.c_float(0)
    _check(load().cj_choose_tile(kernel, ctypes.byref(a), batch, steps, out.ctypes.data, ctypes.byref(pred)),
           "cj_choose_tile")
    return tuple(int(v) for v in out), pred.value

