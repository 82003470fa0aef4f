"""C-ABI checks that need no GPU: exports, keys, dispatch, errors, the
background compile thread and the no-file-system rule (Sec. 1, Sec. 4).

libcj is initialised in compile-only mode: NVRTC compiles to sm_103a CUBIN
on the host, nothing is loaded or launched."""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1904_08555_b300 import cj


def header_functions():
    with open(os.path.join(ROOT, "include", "cj.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:cj_status|const char \*)\s*(cj_\w+)\(", text, re.M)))


def exported_symbols():
    out = subprocess.run(["nm", "-D", "--defined-only", cj.lib_path()], capture_output=True, text=True).stdout
    return sorted(l.split()[-1] for l in out.splitlines() if l.split()[-1].startswith("cj_"))


def test_library_exports_exactly_the_header():
    cj.load()
    assert header_functions() == exported_symbols()
    assert set(header_functions()) == set(cj.EXPORTS)


@pytest.fixture
def compile_only_sync():
    cj.init(compile_only=True, sync=True)
    yield
    cj.shutdown()


def golden_requests():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "keys.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            v = line.split()
            rows.append(([int(x) for x in v[:12]], v[12], int(v[13])))
    return rows


def test_golden_keys_and_dispatch(compile_only_sync):
    """Requests that name their tile: the key and the variant are the
    golden ones, bit for bit."""
    for (k, dt, n, la, lb, m, d, t0, t1, t2, t3, fl), key, var in golden_requests():
        h = cj.specialize(k, dt, n, la, lb, m, d, (t0, t1, t2, t3), fl, allow_compile_error=True)
        got_key, got_var = h.info()
        assert got_key == key, (k, dt, n, la, lb, fl)
        expect = var
        if fl & cj.FLAG_INJECT_COMPILE_ERROR:
            expect = 0      # failed compiles keep the generic kernel
        assert got_var == expect, (k, dt, n, la, lb, fl)


DEFAULT_TILE_REQUESTS = [
    # kernel, dtype, n, layout_a, layout_b, m, d, flags
    (cj.K_UPDATE_CHAIN, cj.F64, n, la, 0, 0, 0, 0) for n in (1, 3, 4, 5, 8, 12, 16, 32, 40, 64) for la in (0, 1)
] + [
    (cj.K_UPDATE_CHAIN, cj.F32, n, 0, 0, 0, 0, 0) for n in (2, 4, 7, 9, 16, 24, 32, 48, 64)
] + [
    (cj.K_UPDATE_CHAIN, cj.BF16, n, 0, 0, 0, 0, 0) for n in (16, 40, 64)
] + [
    (cj.K_UPDATE_CHAIN, cj.F64, 8, 0, 0, 0, 0, cj.FLAG_NO_AOT),
    (cj.K_UPDATE_CHAIN, cj.F32, 16, 1, 0, 0, 0, cj.FLAG_NO_AOT),
] + [
    (cj.K_UPDATE_CHAIN_GROUPED, dt, n, 0, 0, 0, 0, 0) for dt in (cj.F64, cj.F32) for n in (2, 9, 17, 64)
] + [
    (cj.K_UPDATE_CHAIN_GROUPED, cj.BF16, n, 0, 0, 0, 0, 0) for n in (16, 48)
] + [
    (cj.K_LTIMES, dt, 0, la, lb, 36, 96, 0) for dt in (cj.F64, cj.F32) for la, lb in ((0, 0), (1, 3), (4, 2), (5, 5))
] + [
    (cj.K_LTIMES, cj.F32, 0, 0, 1, 64, 128, 0),
    (cj.K_LTIMES, cj.F32, 0, 2, 4, 48, 100, 0),
    (cj.K_LPLUSTIMES, cj.F32, 0, 1, 2, 36, 96, 0),
    (cj.K_LPLUSTIMES, cj.F64, 0, 3, 0, 36, 96, 0),
] + [
    (cj.K_EIGEN_RECURRENCE, dt, n, 0, 0, 0, 0, 0) for dt in (cj.F64, cj.F32) for n in (1, 2, 8, 16, 31)
]


def test_default_tile_requests_resolve_to_a_candidate(compile_only_sync):
    """Requests that leave the tile to the library (tile 0, no cost model):
    the tile the library resolves is one of the request's candidates
    (cj_candidates), the handle's key is the canonical key of the request
    with that tile (every other field bit for bit), and the variant follows
    the contract's rule (ahead-of-time kernel for the f64/f32 update chain at
    n in {4, 8, 16, 32}, else a run-time compile).  Which candidate the
    default rule picks is the library's performance choice and is not
    restated here."""
    from oracle import keys as K
    for (k, dt, n, la, lb, m, d, fl) in DEFAULT_TILE_REQUESTS:
        h = cj.specialize(k, dt, n, la, lb, m, d, (0, 0, 0, 0), fl)
        key_hex, var = h.info()
        tile = K.parse_key(bytes.fromhex(key_hex))["tile"]
        assert tile in cj.candidates(k, dt, n, la, lb, m, d), (k, dt, n, la, lb, tile)
        assert key_hex == K.canonical_key(k, dt, n, la, lb, m, d, tile, fl).hex(), (k, dt, n, la, lb)
        assert var == K.expected_variant(k, dt, n, True, fl), (k, dt, n, la, lb, fl)


def test_explicit_resolved_tile_is_the_same_instantiation(compile_only_sync):
    """A request naming the tile that a default request resolved to has the
    same key, so the cache returns the same handle: at the ahead-of-time
    sizes that is the ahead-of-time kernel (an explicit specialization wins,
    Sec. 2); any other candidate is a different instantiation, compiled at
    run time."""
    from oracle import keys as K
    for dt in (cj.F64, cj.F32):
        for n in K.AOT_SIZES:
            h0 = cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n)
            assert h0.variant == "aot"
            tile = K.parse_key(bytes.fromhex(h0.key_hex))["tile"]
            assert cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n, tile=tile) == h0
            other = next(t for t in cj.candidates(cj.K_UPDATE_CHAIN, dt, n=n) if t != tile)
            h1 = cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n, tile=other)
            assert h1 != h0 and h1.variant == "jit"
            assert h1.key_hex == K.canonical_key(K.K_UPDATE_CHAIN, dt, n, tile=other).hex()
    s = cj.stats()
    assert s["aot_hits"] == 8 and s["cache_hits"] >= 8


def test_cache_returns_same_handle(compile_only_sync):
    a = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=5)
    b = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=5)
    c = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=5, m=7, d=3)     # unused fields ignored
    assert a == b == c
    s = cj.stats()
    assert s["requests"] == 3 and s["cache_hits"] == 2 and s["compiles_ok"] == 1


def test_aot_sizes_are_not_compiled(compile_only_sync):
    for n in (4, 8, 16, 32):
        for dt in (cj.F64, cj.F32):
            assert cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n).variant == "aot"
    s = cj.stats()
    assert s["compiles_ok"] == 0 and s["aot_hits"] == 8


@pytest.mark.parametrize("kw", [
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=0),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=65),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=4, layout_a=2),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=5, n=4),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=12, tile=(2, 64, 0, 0)),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F32, n=16, tile=(4, 2, 0, 0)),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=12, tile=(4, 2, 0, 0)),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=40, tile=(4, 1, 0, 0)),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=8, flags=0x40),
    dict(kernel=cj.K_LTIMES, dtype=cj.F64, layout_a=6, m=36, d=96),
    dict(kernel=cj.K_LTIMES, dtype=cj.F64, m=0, d=96),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 128, 97, (4 << 8) | 12)),
    dict(kernel=cj.K_LTIMES, dtype=cj.BF16, m=36, d=96),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 64, 128, (1 << 16) | (2 << 8) | 8)),
    dict(kernel=cj.K_LTIMES, dtype=cj.F64, m=36, d=95, tile=(1, 64, 128, (1 << 16) | (2 << 8) | 8)),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 128, 320, (3 << 16) | (2 << 8) | 6)),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 128, 64, (3 << 16) | (2 << 8) | 36)),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 128, 128, (3 << 16) | (2 << 8) | 12)),
    dict(kernel=cj.K_LTIMES, dtype=cj.F64, m=36, d=96, tile=(1, 128, 192, (3 << 16) | (2 << 8) | 12)),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=8, flags=0x200),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, flags=0x200 | 0x1),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, m=36, d=96, tile=(1, 64, 96, (1 << 20) | (2 << 8) | 12), flags=0x200),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.F64, n=33),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.BF16, n=8),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.F64, n=8, tile=(2, 4, 0, 0)),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.F64, n=8, tile=(1, 200, 0, 0)),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.F32, n=32, tile=(2, 200, 0, 0)),
    dict(kernel=cj.K_EIGEN_RECURRENCE, dtype=cj.F32, n=8, tile=(3, 4, 0, 0)),
    dict(kernel=9, dtype=cj.F64, n=4),
])
def test_invalid_arguments(compile_only_sync, kw):
    with pytest.raises(cj.CJError) as e:
        cj.specialize(**kw)
    assert e.value.status == cj.CJ_ERR_INVALID_ARG
    assert cj.last_error()


def test_not_initialised_and_launch_without_device():
    with pytest.raises(cj.CJError) as e:
        cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=4)
    assert e.value.status == cj.CJ_ERR_NOT_INITIALIZED
    cj.init(compile_only=True, sync=True)
    try:
        h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=4)
        with pytest.raises(cj.CJError) as e:
            cj.launch_update_chain(h, 1 << 20, 2 << 20, 10, batch=4)
        assert e.value.status == cj.CJ_ERR_NO_DEVICE
        with pytest.raises(cj.CJError) as e:
            cj.launch_update_chain(h, 1 << 20, 2 << 20, 10, batch=-1)
        assert e.value.status == cj.CJ_ERR_INVALID_ARG
    finally:
        cj.shutdown()


def test_compile_failure_reports_log_and_keeps_generic(compile_only_sync):
    with pytest.raises(cj.CJError) as e:
        cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=6, flags=cj.FLAG_INJECT_COMPILE_ERROR)
    assert e.value.status == cj.CJ_ERR_COMPILE
    assert "this_identifier_does_not_exist" in cj.last_error()
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=6, flags=cj.FLAG_INJECT_COMPILE_ERROR,
                      allow_compile_error=True)
    assert h.variant == "generic"
    assert cj.stats()["compiles_failed"] == 1


def test_async_compile_and_wait():
    cj.init(compile_only=True, sync=False, compile_threads=2)
    try:
        hs = [cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n) for n in (5, 6, 7)]
        assert hs[0].wait(0) in (cj.CJ_ERR_TIMEOUT, cj.CJ_OK)
        for h in hs:
            assert h.wait(-1) == cj.CJ_OK
            assert h.variant == "jit"
        bad = cj.specialize(cj.K_LTIMES, cj.F64, m=4, d=4, flags=cj.FLAG_INJECT_COMPILE_ERROR)
        assert bad.wait(-1) == cj.CJ_ERR_COMPILE
        assert bad.variant == "generic"
        s = cj.stats()
        assert s["compiles_ok"] == 3 and s["compiles_failed"] == 1
        assert s["compile_ms_p50"] > 0
    finally:
        cj.shutdown()


NOFS_PROG = """
import ctypes, sys
sys.path.insert(0, {root!r})
from paper_1904_08555_b300 import cj
shim = ctypes.CDLL(None)
shim.shim_log.restype = ctypes.c_char_p
cj.init(compile_only=True, sync=True)
shim.shim_arm(1)
h1 = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=11)
h2 = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=3, layout_b=1, m=36, d=96)
h3 = cj.specialize(cj.K_UPDATE_CHAIN_GROUPED, cj.F32, n=20)
shim.shim_arm(0)
print("COUNT", shim.shim_count())
print("LOG", shim.shim_log().decode().replace(chr(10), ";"))
print("VARIANTS", h1.variant, h2.variant, h3.variant)
"""


def _run_nofs(tmp_path, unset_pwd):
    shim = tmp_path / "nofs_shim.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-o", str(shim),
                    os.path.join(ROOT, "tests", "support", "nofs_shim.c"), "-ldl"], check=True)
    env = dict(os.environ, LD_PRELOAD=str(shim))
    if unset_pwd:
        env.pop("PWD", None)
    else:
        env["PWD"] = os.getcwd()
    r = subprocess.run([sys.executable, "-c", NOFS_PROG.format(root=ROOT)], capture_output=True, text=True,
                       env=env, timeout=300, cwd=os.getcwd())
    assert r.returncode == 0, r.stderr
    out = dict(l.split(" ", 1) for l in r.stdout.splitlines() if l.split(" ", 1)[0] in ("COUNT", "LOG", "VARIANTS"))
    assert out["VARIANTS"] == "jit jit jit"
    calls = [c for c in out.get("LOG", "").split(";") if c]
    return int(out["COUNT"]), calls


def test_no_file_system_access_during_compiles(tmp_path):
    """Three JIT compiles after cj_init open, read, stat or dlopen nothing."""
    count, calls = _run_nofs(tmp_path, unset_pwd=True)
    assert count == 0, calls


def test_compiles_open_no_file_when_pwd_is_set(tmp_path):
    """With $PWD set, NVRTC's current-directory query stats $PWD and "."
    (two metadata calls per compile); no file is opened or read."""
    count, calls = _run_nofs(tmp_path, unset_pwd=False)
    assert all(c.split()[0] in ("stat", "lstat") for c in calls), calls
    assert {c.split(" ", 1)[1] for c in calls} <= {".", os.getcwd()}, calls


@pytest.mark.parametrize("req", [
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=3),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=16),
    dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F32, n=64),
    dict(kernel=cj.K_LTIMES, dtype=cj.F64, layout_a=1, layout_b=3, m=36, d=96),
    dict(kernel=cj.K_LTIMES, dtype=cj.F32, layout_a=4, layout_b=0, m=36, d=96),
])
def test_every_candidate_tile_is_a_valid_request(compile_only_sync, req):
    k = req.pop("kernel")
    cands = cj.candidates(k, **req)
    assert 2 <= len(cands) <= 16
    assert len(set(cands)) == len(cands)
    for tile in cands[:3]:
        h = cj.specialize(k, tile=tile, **req)      # compiles in compile-only mode
        assert h.variant in ("jit", "aot")         # the default tile may be an AoT kernel
    default = cj.specialize(k, **req)             # tile 0: the library's default rule
    dkey = bytes.fromhex(default.key_hex)
    dtile = tuple(int.from_bytes(dkey[12 + 4 * i:16 + 4 * i], "little") for i in range(4))
    assert dtile in cands                          # the default rule's tile is always searched
    for tile in cands:
        f = cj.featurize(k, batch=1 << 16, steps=64, tile=tile, **req)
        assert f.shape == (cj.FEATURES,) and np.all(np.isfinite(f))
        assert f[31] == (1.0 if tuple(tile) == dtile else 0.0)   # flags the default rule's tile


def test_eigen_tile_features_follow_the_thread_mapping(compile_only_sync):
    """Eigen recurrence tiles are featurized by their thread shape: mapping 1
    like the chain's one row per thread, mapping 2 like its two rows per
    thread (chain mapping 6), with the block's real thread count."""
    import math
    for n in (5, 16, 31):
        kw = dict(batch=4096, steps=64, n=n)
        e1 = cj.featurize(cj.K_EIGEN_RECURRENCE, cj.F32, tile=(1, 4, 0, 0), **kw)
        e2 = cj.featurize(cj.K_EIGEN_RECURRENCE, cj.F32, tile=(2, 4, 0, 0), **kw)
        c1 = cj.featurize(cj.K_UPDATE_CHAIN, cj.F32, tile=(1, 4, 0, 0), **kw)
        c6 = cj.featurize(cj.K_UPDATE_CHAIN, cj.F32, tile=(6, 4, 0, 0), **kw)
        assert e2[21] == 0 and e2[20] == 1 and e2[19] == 0.5
        assert math.isclose(float(e2[24]), math.log2(((4 * ((n + 1) // 2) + 31) // 32) * 32) / 10, rel_tol=1e-6)
        np.testing.assert_array_equal(e1[19:25], c1[19:25])
        np.testing.assert_array_equal(e2[19:25], c6[19:25])


def test_plain_c_client(tmp_path):
    """The boundary is C: include/cj.h compiles as C99 with every warning an
    error, and a C program linked against libcj.so initialises it
    (compile-only), specializes, reads the key and stats, sees an
    out-of-range request refused, and shuts down."""
    from oracle import keys as K
    cj.load()
    exe = tmp_path / "c_client"
    libdir = os.path.dirname(cj.lib_path())
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "support", "c_client.c"),
                    cj.lib_path(), "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    key, variant, refused, requests, compiles_ok = r.stdout.split()
    tile = K.parse_key(bytes.fromhex(key))["tile"]
    assert key == K.canonical_key(K.K_UPDATE_CHAIN, K.F64, n=12, tile=tile).hex()
    assert tile in cj.candidates(cj.K_UPDATE_CHAIN, cj.F64, n=12)
    assert int(variant) == K.expected_variant(K.K_UPDATE_CHAIN, K.F64, 12, True) == K.VARIANT_JIT
    assert int(refused) == cj.CJ_ERR_INVALID_ARG
    assert int(requests) >= 1 and int(compiles_ok) >= 1


def test_lplustimes_keys_and_compiles(compile_only_sync):
    from oracle import keys as K
    h = cj.specialize(cj.K_LPLUSTIMES, cj.F64, layout_a=3, layout_b=1, m=36, d=96)
    tile = K.parse_key(bytes.fromhex(h.key_hex))["tile"]
    assert h.key_hex == K.canonical_key(K.K_LPLUSTIMES, K.F64, layout_a=3, layout_b=1, m=36, d=96, tile=tile).hex()
    assert h.variant == "jit"
    assert cj.specialize(cj.K_LPLUSTIMES, cj.F32, layout_a=0, layout_b=5, m=36, d=96).variant == "jit"
    assert len(cj.candidates(cj.K_LPLUSTIMES, cj.F32, layout_a=0, layout_b=5, m=36, d=96)) >= 4


def test_wait_timeout_hook_is_part_of_the_key(compile_only_sync):
    """The hook compiles a different kernel (its own key) and only for the
    tensor-core tiles; the default FP32 LTimes tile is one."""
    plain = cj.specialize(cj.K_LTIMES, cj.F32, m=36, d=96)
    hooked = cj.specialize(cj.K_LTIMES, cj.F32, m=36, d=96, flags=cj.FLAG_INJECT_WAIT_TIMEOUT)
    kp, kh = bytes.fromhex(plain.key_hex), bytes.fromhex(hooked.key_hex)
    assert kp[:28] == kh[:28] and kh[28:] == (0x200).to_bytes(4, "little") and kp[28:] == bytes(4)
    assert hooked.variant == "jit"


def test_vectorised_ltimes_tiles_reject_misaligned_tensors(compile_only_sync):
    """Tile modes 3-6 move in/out in 16-byte vectors: a misaligned pointer is
    refused before any device work (pointer values only, nothing is read)."""
    h = cj.specialize(cj.K_LTIMES, cj.F32, m=36, d=96)           # default f32 tile: mode 6
    assert (h.info()[0] and ((int.from_bytes(bytes.fromhex(h.key_hex)[24:28], "little") >> 16) & 0xF) == 6)
    for in_ptr, out_ptr in ((1 << 20) + 4, 1 << 21), ((1 << 20), (1 << 21) + 8):
        with pytest.raises(cj.CJError) as e:
            cj.launch_ltimes(h, 1 << 19, in_ptr, out_ptr, 8, 64)
        assert e.value.status == cj.CJ_ERR_INVALID_ARG and "16-byte" in cj.last_error()
    with pytest.raises(cj.CJError) as e:                         # aligned: reaches the device check
        cj.launch_ltimes(h, 1 << 19, 1 << 20, 1 << 21, 8, 64)
    assert e.value.status == cj.CJ_ERR_NO_DEVICE


def test_eigen_recurrence_requests(compile_only_sync):
    """Kernel 5 compiles for n = 1..32 in f64 and f32 (a sample), its key zeroes
    the unused fields, and its candidates are all valid requests."""
    for n in (1, 2, 7, 16, 32):
        for dt in (cj.F64, cj.F32):
            h = cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, layout_a=1, m=5, d=7)
            key = bytes.fromhex(h.key_hex)
            assert key[3:5] == bytes(2) and key[8:12] == bytes(4) and h.variant == "jit"
            for tile in cj.candidates(cj.K_EIGEN_RECURRENCE, dt, n=n):
                cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, tile=tile)


def test_exit_without_shutdown_while_compiling():
    """A process that exits with a run-time compile still in flight and never
    calls cj_shutdown exits cleanly: the library stops its compile threads at
    exit, before the statically linked compiler's own state is torn down."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1904_08555_b300 import cj\n"
            "cj.init(compile_only=True, compile_threads=2)\n"
            "cj.specialize(cj.K_LTIMES, cj.F32, layout_a=0, layout_b=1, m=64, d=128)\n"
            "cj.specialize(cj.K_UPDATE_CHAIN, cj.F32, n=61)\n"
            "print('exiting')\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    assert "exiting" in r.stdout


def test_concurrent_requests_share_one_cache_entry():
    """The cache is program-global: eight host threads requesting the same
    instantiations at once (ctypes drops the GIL for the call) get one handle
    per distinct request, each key equal to the request's canonical key, and
    each distinct request compiled once."""
    import threading
    from oracle import keys as K
    cj.init(compile_only=True, compile_threads=4)
    try:
        reqs = [(cj.K_UPDATE_CHAIN, cj.F64, n, 0, 0, 0, 0) for n in (3, 5, 7, 9, 12, 17, 24)] + \
               [(cj.K_UPDATE_CHAIN, cj.F32, n, 1, 0, 0, 0) for n in (6, 10, 40)] + \
               [(cj.K_LTIMES, cj.F64, 0, la, lb, 36, 96) for la, lb in ((0, 0), (2, 5), (4, 1))]
        got = [dict() for _ in range(8)]
        errors = []
        start = threading.Barrier(8)

        def worker(t):
            try:
                start.wait()
                order = reqs[t % len(reqs):] + reqs[:t % len(reqs)]   # every thread in its own order
                for r in order:
                    got[t][r] = cj.specialize(*r)
            except Exception as e:   # reported below
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors, errors
        for r in reqs:
            hs = {got[t][r].ptr for t in range(8)}
            assert len(hs) == 1, r
            h = got[0][r]
            assert h.wait() == cj.CJ_OK
            tile = K.parse_key(bytes.fromhex(h.key_hex))["tile"]
            k, dt, n, la, lb, m, d = r
            assert h.key_hex == K.canonical_key(k, dt, n, la, lb, m, d, tile, 0).hex(), r
        s = cj.stats()
        assert s["requests"] == 8 * len(reqs)
        assert s["compiles_ok"] + s["compiles_failed"] == len(reqs)
        assert s["cache_hits"] == 8 * len(reqs) - len(reqs)
    finally:
        cj.shutdown()


NEW_TILE_CASES = [
    # (kernel, dtype, n, la, lb, m, d, tile, valid)
    (cj.K_LTIMES, cj.F32, 0, 0, 0, 36, 96, (1, 128, 320, (6 << 20) | (6 << 16) | (4 << 8) | 4), True),
    (cj.K_LTIMES, cj.F32, 0, 3, 5, 64, 64, (1, 128, 448, (4 << 20) | (6 << 16) | (6 << 8) | 8), True),
    (cj.K_LTIMES, cj.F32, 0, 0, 0, 64, 64, (1, 128, 448, (4 << 20) | (6 << 16) | (7 << 8) | 8), False),  # 576 TMEM cols
    (cj.K_LTIMES, cj.F32, 0, 0, 0, 36, 96, (1, 128, 256, (4 << 20) | (6 << 16) | (2 << 8) | 2), False),  # 2 converters
    (cj.K_LTIMES, cj.F64, 0, 0, 0, 36, 96, (1, 128, 320, (6 << 20) | (6 << 16) | (4 << 8) | 4), False),  # f64
    (cj.K_LTIMES, cj.F32, 0, 0, 0, 36, 96, (1, 128, 320, (1 << 20) | (6 << 16) | (4 << 8) | 4), False),  # 1 box
    (cj.K_UPDATE_CHAIN, cj.F32, 33, 0, 0, 0, 0, (8, 3, 0, 0), True),
    (cj.K_UPDATE_CHAIN_GROUPED, cj.F32, 64, 0, 0, 0, 0, (8, 2, 0, 0), True),
    (cj.K_UPDATE_CHAIN, cj.F64, 33, 0, 0, 0, 0, (8, 3, 0, 0), False),   # mapping 8 is f32
    (cj.K_UPDATE_CHAIN, cj.F32, 7, 0, 0, 0, 0, (8, 3, 0, 0), False),    # n >= 8
    (cj.K_UPDATE_CHAIN, cj.F32, 33, 0, 0, 0, 0, (9, 3, 0, 0), False),   # no mapping 9
    (cj.K_MASS, cj.F32, 4, 0, 0, 6, 2, (128, 2, 0, 0), True),
    (cj.K_MASS, cj.F64, 5, 0, 0, 8, 3, (4, 1, 0, 0), True),
    (cj.K_MASS, cj.F64, 4, 0, 0, 6, 3, (128, 2, 0, 0), False),          # form 2 is 2-D
    (cj.K_MASS, cj.F64, 6, 0, 0, 10, 2, (128, 2, 0, 0), False),         # D Q + D^2 = 96 > 80
    (cj.K_MASS, cj.F64, 4, 0, 0, 6, 2, (128, 3, 0, 0), False),          # no form 3
]


@pytest.mark.parametrize("case", NEW_TILE_CASES)
def test_tensor_memory_register_block_and_mass_form_tiles(compile_only_sync, case):
    """LTimes mode 6 (operands in tensor memory), chain mapping 8 (4 x 8 register
    blocks) and the mass operator's forms 1 and 2: valid tiles compile (run-time
    instantiations), invalid ones are refused before any compile."""
    k, dt, n, la, lb, m, d, tile, valid = case
    if valid:
        h = cj.specialize(k, dt, n, la, lb, m, d, tile)
        assert h.variant == "jit"
    else:
        with pytest.raises(cj.CJError) as e:
            cj.specialize(k, dt, n, la, lb, m, d, tile)
        assert e.value.status == cj.CJ_ERR_INVALID_ARG


def test_every_candidate_space_has_at_most_16_tiles(compile_only_sync):
    """The autotuner's variant space V(kernel, dtype) holds at most 16 tiles for
    every request shape: the chains at every n and dtype, LTimes and
    LPlusTimes at every pair of storage orders, the mass operator at every
    dimension, D and Q up to 8."""
    sizes = []
    for dt in (cj.F64, cj.F32, cj.BF16):
        for n in range(16 if dt == cj.BF16 else 1, 65):
            for k in (cj.K_UPDATE_CHAIN, cj.K_UPDATE_CHAIN_GROUPED):
                sizes.append(((k, dt, n), len(cj.candidates(k, dt, n=n))))
    for dt in (cj.F64, cj.F32):
        for la in range(6):
            for lb in range(6):
                for k in (cj.K_LTIMES, cj.K_LPLUSTIMES):
                    sizes.append(((k, dt, la, lb), len(cj.candidates(k, dt, layout_a=la, layout_b=lb, m=36, d=96))))
    for dt in (cj.F64, cj.F32):
        for dim in (2, 3):
            for D in range(1, 9):
                for Q in range(1, 9):
                    sizes.append(((cj.K_MASS, dt, dim, D, Q), len(cj.candidates(cj.K_MASS, dt, n=D, m=Q, d=dim))))
    bad = [(req, c) for req, c in sizes if not 1 <= c <= 16]
    assert not bad, bad[:10]


def test_features_tell_the_new_forms_apart(compile_only_sync):
    """The cost model sees which form a tile is: LTimes mode 6 (operands in
    tensor memory) against mode 5 (the same TMA-fed tile, operands in shared
    memory), and chain mapping 8 (4 x 8 register blocks, columns padded to
    8) against mapping 5 (4 x 4)."""
    import numpy as np
    t5 = (1, 128, 448, (4 << 20) | (5 << 16) | (2 << 8) | 8)
    t6 = (1, 128, 448, (4 << 20) | (6 << 16) | (2 << 8) | 8)
    f5 = cj.featurize(cj.K_LTIMES, cj.F32, 1 << 23, 1, t5, m=36, d=96)
    f6 = cj.featurize(cj.K_LTIMES, cj.F32, 1 << 23, 1, t6, m=36, d=96)
    assert f5[2] == f6[2] == 1.0            # both tensor-core tiles
    assert f5[5] == f6[5] == 1.0            # both fed by TMA
    assert f5[25] != f6[25]                 # the mode itself
    assert np.count_nonzero(f5 != f6) >= 1
    g5 = cj.featurize(cj.K_UPDATE_CHAIN, cj.F32, 1 << 14, 64, (5, 1, 0, 0), n=60)
    g8 = cj.featurize(cj.K_UPDATE_CHAIN, cj.F32, 1 << 14, 64, (8, 1, 0, 0), n=60)
    assert g5[22] == g8[22] == 1.0          # register-blocked panels
    assert g5[19] != g8[19]                 # 4 x 4 against 4 x 8
    assert g8[12] > g5[12] >= 0.0           # padding: n = 60 is a multiple of 4, not of 8


def test_binding_refuses_tensors_that_do_not_fit(compile_only_sync):
    """The launch wrappers check each tensor against the request before calling
    into libcj: a contiguous CUDA tensor of the handle's element type holding
    enough elements.  Here (no GPU) every tensor is a host tensor, so each call
    is refused with CJ_ERR_INVALID_ARG and never reaches the launch."""
    torch = pytest.importorskip("torch")
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=4)
    A = torch.zeros(3, 4, 4, dtype=torch.float64)
    with pytest.raises(cj.CJError) as e:
        cj.launch_update_chain(h, A, A, 8)
    assert e.value.status == cj.CJ_ERR_INVALID_ARG and "CUDA" in str(e.value)
    hl = cj.specialize(cj.K_LTIMES, cj.F32, m=36, d=96)
    small = torch.zeros(10, dtype=torch.float32)
    with pytest.raises(cj.CJError) as e:
        cj.launch_ltimes(hl, small, small, small, 8, 64)
    assert e.value.status == cj.CJ_ERR_INVALID_ARG
    hm = cj.specialize(cj.K_MASS, cj.F64, n=3, m=4, d=2)
    with pytest.raises(cj.CJError):
        cj.launch_mass(hm, small, small, small, small, 5)
    # an empty batch reads and writes nothing: no check, and libcj answers (no device here)
    with pytest.raises(cj.CJError) as e:
        cj.launch_mass(hm, small, small, small, small, 0)
    assert e.value.status == cj.CJ_ERR_NO_DEVICE
