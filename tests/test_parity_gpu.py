"""GPU parity: libcj kernels (through the C ABI) against the CPU oracle.

FP64 tolerance: 1e-12 relative Frobenius error per instance (update chain;
max over instances) and over the whole output (LTimes).  FP32 variants are
gated at 1e-5 against the FP64 oracle.  Sizes span several blocks and end in
ragged tails; full-size launches are checked on seeded samples.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True, compile_threads=2)
    yield
    cj.shutdown()


def relF_per_instance(x, ref):
    x = x.reshape(ref.shape[0], -1).astype(np.float64)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def tdtype(dt):
    return torch.float64 if dt == cj.F64 else torch.float32


def run_chain(h, A_np, steps, dt):
    A = torch.from_numpy(A_np).to("cuda", tdtype(dt))
    X = torch.full_like(A, float("nan"))
    cj.launch_update_chain(h, A, X, steps)
    torch.cuda.synchronize()
    return X.cpu().numpy()


def oracle_batch(n, steps):
    return int(np.clip(3e7 // (n ** 3 * steps), 5, 700))


CHAIN_SIZES = [1, 2, 3, 4, 5, 7, 8, 12, 16, 24, 31, 32, 33, 48, 64]


@pytest.mark.parametrize("n", CHAIN_SIZES)
@pytest.mark.parametrize("variant", ["default", "generic", "no_aot"])
def test_update_chain_f64(n, variant):
    steps = 64
    flags = {"default": 0, "generic": cj.FLAG_GENERIC, "no_aot": cj.FLAG_NO_AOT}[variant]
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=flags)
    expect = {"generic": "generic", "no_aot": "jit"}.get(variant, "aot" if n in (4, 8, 16, 32) else "jit")
    assert h.variant == expect
    batch = oracle_batch(n, steps) + 3
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    ref = oracle.update_chain(A, steps, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F64), ref) <= TOL64


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 16, 40])
@pytest.mark.parametrize("steps", [1, 100])
def test_update_chain_col_major(n, steps):
    for flags in (0, cj.FLAG_GENERIC):
        h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, layout_a=1, flags=flags)
        batch = oracle_batch(n, steps) + 1
        A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=1)
        ref = oracle.update_chain(A, steps, layout=1, nthreads=8)
        assert relF_per_instance(run_chain(h, A, steps, cj.F64), ref) <= TOL64


@pytest.mark.parametrize("n,tile", [(3, (2, 32, 0, 0)), (5, (2, 128, 0, 0)), (8, (2, 64, 0, 0)),
                                    (8, (1, 1, 0, 0)), (12, (1, 3, 0, 0)), (24, (1, 16, 0, 0)),
                                    (64, (1, 1, 0, 0)), (40, (1, 5, 0, 0))])
def test_update_chain_explicit_tiles(n, tile):
    steps = 32
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, tile=tile)
    assert h.variant == "jit"
    batch = oracle_batch(n, steps) + 7
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    ref = oracle.update_chain(A, steps, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F64), ref) <= TOL64


@pytest.mark.parametrize("n", [8, 16, 24, 32])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("ipb", [1, 3])
def test_update_chain_fp64_tensor_core_tiles(n, layout, ipb):
    """Mapping 4 (mma.sync m8n8k4 panels) against the oracle and against the
    FMA-pipe mapping 1 on the same inputs."""
    steps = 64
    batch = oracle_batch(n, steps) + 5
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    h4 = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, layout_a=layout, tile=(4, ipb, 0, 0))
    h1 = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, layout_a=layout, tile=(1, 8, 0, 0))
    x4 = run_chain(h4, A, steps, cj.F64)
    x1 = run_chain(h1, A, steps, cj.F64)
    assert relF_per_instance(x4, ref) <= TOL64
    assert relF_per_instance(x1, ref) <= TOL64
    assert relF_per_instance(x4, x1) <= TOL64


@pytest.mark.parametrize("n,ipb", [(8, 8), (12, 4), (16, 3), (32, 2), (48, 1), (64, 1),
                                   (9, 4), (13, 3), (30, 2), (45, 1), (61, 1), (63, 2)])
@pytest.mark.parametrize("layout", [0, 1])
def test_update_chain_f32_register_blocks(n, ipb, layout):
    """Mapping 5 (4x4 register blocks, X transposed in shared memory); n not a
    multiple of 4 runs padded with zeros."""
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F32, n=n, layout_a=layout, tile=(5, ipb, 0, 0))
    batch = oracle_batch(n, steps) + 2
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("n,ipb", [(8, 4), (16, 4), (17, 2), (24, 3), (30, 2), (32, 5), (33, 2), (45, 1),
                                   (48, 2), (61, 1), (63, 2), (64, 1), (64, 3)])
@pytest.mark.parametrize("layout", [0, 1])
def test_update_chain_f32_register_blocks_4x8(n, ipb, layout):
    """Mapping 8 (4 x 8 register blocks: rows padded to 4, columns to 8 with
    zeros, X transposed in shared memory), ragged last block."""
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F32, n=n, layout_a=layout, tile=(8, ipb, 0, 0))
    assert h.variant == "jit"
    batch = oracle_batch(n, steps) + 2
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("n,ipb", [(2, 32), (5, 16), (7, 9), (8, 8), (12, 4), (15, 5), (16, 3), (31, 2), (32, 8)])
@pytest.mark.parametrize("layout", [0, 1])
def test_update_chain_f32_two_rows_per_thread(n, ipb, layout):
    """Mapping 6 (rows h and h + ceil(n/2) per thread; odd n leaves the last
    thread's second row empty), ragged last block."""
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F32, n=n, layout_a=layout, tile=(6, ipb, 0, 0))
    batch = oracle_batch(n, steps) + 3
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("n", [3, 8, 16, 32, 48, 64])
@pytest.mark.parametrize("generic", [False, True])
def test_update_chain_f32_error(n, generic):
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F32, n=n, flags=cj.FLAG_GENERIC if generic else 0)
    batch = oracle_batch(n, steps) + 2
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    ref = oracle.update_chain(A, steps, nthreads=8)
    assert relF_per_instance(run_chain(h, A, steps, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("n", [16, 17, 24, 32, 40, 64])
@pytest.mark.parametrize("layout", [0, 1])
def test_update_chain_bf16_error(n, layout):
    """bf16 tensor-core operands, fp32 accumulate and state: reported error
    against the FP64 oracle, gated at 2e-2."""
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.BF16, n=n, layout_a=layout)
    assert h.variant == "jit"
    batch = oracle_batch(n, steps) + 3
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    err = relF_per_instance(run_chain(h, A, steps, cj.F32), ref)
    print(f"bf16 n={n} layout={layout} max rel-F error {err:.3e}")
    assert err <= 2e-2
    assert err > 1e-7       # operands really are rounded to bf16


@pytest.mark.parametrize("n", [16, 17, 24, 31, 32, 33, 48, 63, 64])
@pytest.mark.parametrize("layout", [0, 1])
def test_update_chain_bf16_tcgen05(n, layout):
    """Mapping 7: bf16 operands on tcgen05.mma (accumulator in tensor
    memory), fp32 state in registers, one instance per block at a time over a
    persistent grid; gated at 2e-2 against the FP64 oracle like mapping 3,
    and close to mapping 3's own result (both round the same operands)."""
    steps = 64
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.BF16, n=n, layout_a=layout, tile=(7, 1, 0, 0))
    assert h.variant == "jit"
    batch = oracle_batch(n, steps) + 3
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n, layout=layout)
    ref = oracle.update_chain(A, steps, layout=layout, nthreads=8)
    got = run_chain(h, A, steps, cj.F32)
    assert np.all(np.isfinite(got))
    err = relF_per_instance(got, ref)
    print(f"bf16 tcgen05 n={n} layout={layout} max rel-F error {err:.3e}")
    assert 1e-7 < err <= 2e-2
    h3 = cj.specialize(cj.K_UPDATE_CHAIN, cj.BF16, n=n, layout_a=layout, tile=(3, 1, 0, 0))
    assert relF_per_instance(got, run_chain(h3, A, steps, cj.F32).astype(np.float64)) <= 2e-2


def test_update_chain_bf16_tcgen05_large_batch():
    """More instances than resident blocks: each persistent block runs many
    instances, re-staging its B operand and reusing its tensor memory."""
    n, steps, batch = 64, 40, 4000
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.BF16, n=n, tile=(7, 1, 0, 0))
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    got = run_chain(h, A, steps, cj.F32)
    idx = np.r_[0:5, batch // 2:batch // 2 + 5, batch - 5:batch]
    ref = oracle.update_chain(A[idx], steps, nthreads=8)
    assert relF_per_instance(got[idx], ref) <= 2e-2


def test_small_config_all_variants():
    """64 FP64 matrices, N = 8, T = 100: JIT, AoT and generic all match."""
    A = synth.chain_inputs_np(synth.SEED_CHAIN_SMALL, 64, 8)
    ref = oracle.update_chain(A, 100)
    for flags, var in ((cj.FLAG_NO_AOT, "jit"), (0, "aot"), (cj.FLAG_GENERIC, "generic")):
        h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=8, flags=flags)
        assert h.variant == var
        assert relF_per_instance(run_chain(h, A, 100, cj.F64), ref) <= TOL64


def test_empty_batch_is_a_no_op():
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=5)
    X = torch.full((3, 5, 5), 7.0, device="cuda", dtype=torch.float64)
    cj.launch_update_chain(h, X, X, 10, batch=0)
    torch.cuda.synchronize()
    assert torch.all(X == 7.0)


def test_registers_specialized_vs_generic():
    for n in (2, 4, 7):
        spec = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_NO_AOT)
        gen = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_GENERIC)
        rs, _ = spec.regs()
        rg, _ = gen.regs()
        assert rs > 0 and rg > 0


# ---------------------------------------------------------------------------
# LTimes
# ---------------------------------------------------------------------------

def run_ltimes(h, L, x_canon, lin, lout, dt):
    M, D = L.shape
    _, G, Z = x_canon.shape
    Lt = torch.from_numpy(L).to("cuda", tdtype(dt))
    xt = torch.from_numpy(synth.to_layout(x_canon, lin).ravel()).to("cuda", tdtype(dt))
    out = torch.full((M * G * Z,), float("nan"), device="cuda", dtype=tdtype(dt))
    cj.launch_ltimes(h, Lt, xt, out, G, Z)
    torch.cuda.synchronize()
    return synth.from_layout(out.cpu().numpy(), lout, (M, G, Z)).astype(np.float64)


def relF(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def lt_small():
    M, D, G, Z = 36, 96, 5, 37
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=4).reshape(M, G, Z)
    return L, x, ref


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
def test_ltimes_all_orders_f64(lt_small, lin, lout):
    L, x, ref = lt_small
    h = cj.specialize(cj.K_LTIMES, cj.F64, layout_a=lin, layout_b=lout, m=36, d=96)
    assert h.variant == "jit"
    out = run_ltimes(h, L, x, lin, lout, cj.F64)
    assert relF(out, ref) <= TOL64
    for m in range(36):
        assert relF(out[m], ref[m]) <= TOL64


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", [0, 3, 4])
def test_ltimes_orders_f32(lt_small, lin, lout):
    L, x, ref = lt_small
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", [1, 5])
@pytest.mark.parametrize("tg,tz,pipe", [(1, 64, 1), (8, 16, 0), (32, 4, 1)])
def test_ltimes_f32_tf32x3(lt_small, lin, lout, tg, tz, pipe):
    """3xTF32 tensor-core mode: FP32-level accuracy against the FP64 oracle."""
    L, x, ref = lt_small
    tile = (tg, tz, tg * tz // 16 * 32, (pipe << 20) | (2 << 16) | (1 << 8) | 8)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96, tile=tile)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", [0, 3, 4])
@pytest.mark.parametrize("tg,tz,r", [(1, 256, 2), (8, 16, 1), (32, 8, 2)])
def test_ltimes_f32_direct(lt_small, lin, lout, tg, tz, r):
    """Mode 3: direct global loads of `in`, staged out box (ragged G = 5, Z = 37)."""
    L, x, ref = lt_small
    tile = (tg, tz, tg * tz // r, (3 << 16) | (r << 8))
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96, tile=tile)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
@pytest.mark.parametrize("tg,tz,r,s", [(1, 128, 2, 12), (8, 16, 1, 8), (32, 8, 4, 12)])
def test_ltimes_f32_direct_split_moments(lt_small, lin, lout, tg, tz, r, s):
    """Mode 3 with S moments per thread (S = 8 leaves a partial last group of 4)
    over every storage-order pair: direct and staged stores."""
    L, x, ref = lt_small
    tile = (tg, tz, tg * tz // r * -(-36 // s), (3 << 16) | (r << 8) | s)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96, tile=tile)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32


@pytest.mark.parametrize("M,D,G,Z,lin,lout,tile", [
    (37, 12, 3, 50, 0, 0, (1, 64, 128, (3 << 16) | (2 << 8) | 12)),     # partial group, vector d loads
    (37, 12, 3, 50, 3, 5, (8, 8, 192, (3 << 16) | (1 << 8) | 16)),      # partial group, staged out box
    (9, 7, 4, 33, 1, 4, (32, 4, 128, (3 << 16) | (1 << 8))),            # M not a multiple of 4, scalar d
    (64, 8, 2, 130, 3, 3, (1, 128, 256, (3 << 16) | (1 << 8) | 32)),    # M_FAST direct float4 stores
])
def test_ltimes_f32_direct_shapes(M, D, G, Z, lin, lout, tile):
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D, tile=tile)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32


def tc_tile(lin, lout, stages=2, nprod=8, tg=None):
    """tcgen05 tile (mode 4): 128 columns, box shape by the faster column axes."""
    if tg is None:
        gi, go = lin in (1, 4), lout in (1, 4)
        tg = 1 if not (gi or go) else (8 if (gi and lout in (0, 2)) or (go and lin in (0, 2)) else 32)
    return (tg, 128 // tg, 32 * (5 + nprod), (4 << 16) | (stages << 8) | nprod)


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
@pytest.mark.parametrize("stages,nprod", [(2, 8), (4, 8), (3, 4)])
def test_ltimes_f32_tcgen05(lt_small, lin, lout, stages, nprod):
    """Mode 4: tcgen05.mma kind::tf32 (3xTF32), accumulator in tensor memory,
    every storage-order pair, ragged G = 5, Z = 37."""
    L, x, ref = lt_small
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96,
                      tile=tc_tile(lin, lout, stages, nprod))
    assert h.variant == "jit"
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("lin,lout,tg", [(0, 0, None), (3, 5, None), (4, 1, None), (1, 4, 8), (2, 3, 1), (5, 0, 8)])
def test_ltimes_f32_tcgen05_many_tiles_per_block(lin, lout, tg):
    """2048 tiles over at most one block per SM: both accumulators and every
    stage go through many phases."""
    M, D, G, Z = 36, 96, 32, 8192
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=8).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D, tile=tc_tile(lin, lout, tg=tg))
    out = run_ltimes(h, L, x, lin, lout, cj.F32)
    assert relF(out, ref) <= TOL32
    for m in (0, 17, 35):
        assert relF(out[m], ref[m]) <= TOL32
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("M,D,G,Z,lin,lout,stages,nprod", [
    (36, 96, 6, 44, 4, 5, 4, 8),      # g-fastest in with G % 4 != 0: scalar column loads
    (36, 96, 8, 64, 1, 0, 4, 4),      # g-fastest in, TG = 8 box
    (37, 12, 3, 50, 0, 0, 4, 8),      # one K block, zero-padded d; N = 48
    (9, 7, 4, 33, 1, 4, 2, 2),        # D % 4 != 0, scalar loads; N = 16
    (4, 100, 2, 300, 2, 3, 3, 8),     # four K blocks, ragged; m-fastest out
    (64, 128, 3, 70, 3, 3, 2, 8),     # d-fastest float4 loads; N = 64
    (16, 32, 32, 5, 4, 5, 4, 4),      # g-fastest in, 32-wide g box
])
def test_ltimes_f32_tcgen05_shapes(M, D, G, Z, lin, lout, stages, nprod):
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D,
                      tile=tc_tile(lin, lout, stages, nprod))
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32
    assert h.wait_timeouts() == 0


def tma_tile(lin, lout, boxes=4, stages=2, nconv=8, tg=None):
    """tcgen05 tile fed by TMA (mode 5)."""
    t = tc_tile(lin, lout, stages, nconv, tg)
    return (t[0], t[1], 32 * (6 + nconv), (boxes << 20) | (5 << 16) | (stages << 8) | nconv)


@pytest.fixture(scope="module")
def lt_aligned():
    """G and Z multiples of 4 (TMA-compatible for every order), Z ragged against every box."""
    M, D, G, Z = 36, 96, 8, 200
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=4).reshape(M, G, Z)
    return L, x, ref


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
def test_ltimes_f32_tma(lt_aligned, lin, lout):
    """Mode 5: TMA boxes of `in` -> converter warps -> tcgen05 3xTF32; every
    storage-order pair runs on the TMA path."""
    L, x, ref = lt_aligned
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96, tile=tma_tile(lin, lout))
    before = cj.stats()
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32
    after = cj.stats()
    assert after["launches_tma"] == before["launches_tma"] + 1
    assert after["launches_tma_fallback"] == before["launches_tma_fallback"]
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("lin,lout", [(0, 0), (1, 4), (4, 2), (3, 3), (5, 1), (2, 5)])
def test_ltimes_f32_tma_fallback(lt_small, lin, lout):
    """G = 5, Z = 37 admit no tensor map when g or z is innermost: the launch
    runs the mode-4 twin compiled into the same module; d innermost (D = 96)
    still runs on TMA."""
    L, x, ref = lt_small
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=36, d=96, tile=tma_tile(lin, lout))
    before = cj.stats()
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32
    after = cj.stats()
    d_inner = lin in (3, 5)
    assert after["launches_tma"] - before["launches_tma"] == (1 if d_inner else 0)
    assert after["launches_tma_fallback"] - before["launches_tma_fallback"] == (0 if d_inner else 1)
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("lin,lout,tg", [(0, 0, None), (3, 5, None), (4, 1, None), (1, 4, 8), (2, 3, 1), (5, 0, 8)])
def test_ltimes_f32_tma_many_tiles_per_block(lin, lout, tg):
    M, D, G, Z = 36, 96, 32, 8192
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=8).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D, tile=tma_tile(lin, lout, tg=tg))
    before = cj.stats()["launches_tma"]
    out = run_ltimes(h, L, x, lin, lout, cj.F32)
    assert cj.stats()["launches_tma"] == before + 1
    assert relF(out, ref) <= TOL32
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("M,D,G,Z,lin,lout,boxes,stages,nconv", [
    (37, 12, 4, 52, 0, 0, 4, 2, 8),     # one K block, directions 12..31 from TMA zero fill
    (9, 8, 4, 36, 1, 4, 2, 2, 2),       # g innermost, 32-wide g box
    (4, 100, 4, 300, 2, 3, 3, 3, 4),    # four K blocks, ragged; m-fastest out
    (64, 128, 3, 70, 3, 3, 2, 2, 8),    # d innermost (128-byte swizzle), ragged G and Z
    (16, 40, 12, 24, 5, 2, 2, 2, 8),    # d innermost, D not a multiple of 32
])
def test_ltimes_f32_tma_shapes(M, D, G, Z, lin, lout, boxes, stages, nconv):
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D,
                      tile=tma_tile(lin, lout, boxes, stages, nconv))
    before = cj.stats()["launches_tma"]
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F32), ref) <= TOL32
    assert cj.stats()["launches_tma"] == before + 1
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("lin,lout", [(0, 0), (1, 3), (3, 5), (5, 2)])
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
def test_ltimes_generic(lt_small, lin, lout, dt):
    L, x, ref = lt_small
    h = cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=36, d=96, flags=cj.FLAG_GENERIC)
    assert h.variant == "generic"
    assert relF(run_ltimes(h, L, x, lin, lout, dt), ref) <= (TOL64 if dt == cj.F64 else TOL32)


@pytest.mark.parametrize("M,D,G,Z,lin,lout,tile", [
    (4, 6, 3, 130, 0, 5, (0, 0, 0, 0)),
    (37, 11, 33, 9, 4, 1, (0, 0, 0, 0)),             # partial moment group, ragged G
    (36, 96, 32, 64, 2, 2, (4, 16, 192, (1 << 8) | 12)),
    (36, 96, 32, 64, 1, 4, (32, 2, 64, (1 << 8) | 36)),
    (64, 128, 2, 40, 3, 0, (1, 32, 256, (1 << 8) | 8)),
    (36, 96, 32, 64, 0, 3, (1, 64, 256, (1 << 8) | 9)),                       # FMA pipe, f64
    (36, 96, 32, 64, 4, 5, (32, 2, 256, (1 << 16) | (1 << 8) | 8)),           # tensor cores, R = 1
    (36, 96, 5, 37, 2, 1, (8, 16, 128, (1 << 16) | (4 << 8) | 8)),            # tensor cores, R = 4, ragged
    (40, 8, 3, 100, 5, 0, (1, 64, 128, (1 << 16) | (2 << 8) | 8)),            # M multiple of 8
])
def test_ltimes_shapes_and_tiles(M, D, G, Z, lin, lout, tile):
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F64, layout_a=lin, layout_b=lout, m=M, d=D, tile=tile)
    assert relF(run_ltimes(h, L, x, lin, lout, cj.F64), ref) <= TOL64


# ---------------------------------------------------------------------------
# Grouped plan (uneven batch)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", [cj.F64, cj.F32, cj.BF16])
@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_plan_uneven(dt, use_graph):
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 400)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    ref = oracle.update_chain_uneven(n, t, off, pool)
    plan = cj.GroupPlan(dt, n, t)
    try:
        assert plan.pool_elems == pool.size
        A = torch.from_numpy(pool).to("cuda", tdtype(dt))
        for rep in range(2):          # second launch replays the graph
            X = torch.full_like(A, float("nan"))
            plan.launch(A, X, stream=torch.cuda.current_stream(), use_graph=use_graph)
            torch.cuda.synchronize()
            Xh = X.cpu().numpy().astype(np.float64)
            worst = 0.0
            for k in range(len(n)):
                sl = slice(off[k], off[k] + n[k] * n[k])
                worst = max(worst, relF(Xh[sl], ref[sl]))
            assert worst <= {cj.F64: TOL64, cj.F32: TOL32, cj.BF16: 2e-2}[dt], (rep, worst)
    finally:
        plan.destroy()


@pytest.mark.parametrize("dt", [cj.F64, cj.F32, cj.BF16])
def test_grouped_plan_dispatcher(dt):
    """One persistent launch for the whole uneven batch: the plan's generated
    dispatcher (every group's body in one kernel, cost-ordered tickets), as
    a graph and as a direct launch, then the per-group form of the same plan;
    all against the oracle per instance."""
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN + 1, 500)
    n[:4] = (1, 2, 63, 64)             # the ends of the size range
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN + 1, n)
    A = torch.from_numpy(pool).to("cuda", tdtype(dt))
    ref = oracle.update_chain_uneven(n, t, off, A.double().cpu().numpy(), nthreads=8)
    tol = {cj.F64: TOL64, cj.F32: TOL32, cj.BF16: 2e-2}[dt]
    plan = cj.GroupPlan(dt, n, t)
    try:
        plan.wait()
        d = plan.dispatcher()
        assert d["state"] == "ready" and d["threads"] == 256 and d["tickets"] >= plan.n_groups
        for use_graph, per_group in ((True, False), (False, False), (True, True), (False, True)):
            before = cj.stats()["launches_dispatch"]
            X = torch.full_like(A, float("nan"))
            plan.launch(A, X, use_graph=use_graph, per_group=per_group)
            torch.cuda.synchronize()
            if not use_graph:
                assert cj.stats()["launches_dispatch"] - before == (0 if per_group else 1)
            Xh = X.double().cpu().numpy()
            assert np.all(np.isfinite(Xh)), (use_graph, per_group)
            worst = max(relF(Xh[off[k]:off[k] + n[k] * n[k]], ref[off[k]:off[k] + n[k] * n[k]]) for k in range(len(n)))
            lim = tol if dt != cj.BF16 else 2e-2
            assert worst <= lim, (use_graph, per_group, worst)
            if dt == cj.BF16:   # the n < 16 groups run in FP32
                small = max(relF(Xh[off[k]:off[k] + n[k] * n[k]], ref[off[k]:off[k] + n[k] * n[k]])
                            for k in range(len(n)) if n[k] < 16)
                assert small <= TOL32, (use_graph, per_group, small)
    finally:
        plan.destroy()


@pytest.mark.parametrize("dt", [cj.F64, cj.F32, cj.BF16])
def test_grouped_plan_every_dispatcher_variant(dt):
    """Each dispatcher variant the plan's autotuner may keep (register caps;
    for f32 also the 4 x 8 register-block rule for n >= 16; for bf16 also
    blocks of 128 threads), pinned in turn
    and launched as a graph and directly, against the oracle per instance."""
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN + 2, 400)
    n[:6] = (1, 2, 15, 16, 63, 64)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN + 2, n)
    A = torch.from_numpy(pool).to("cuda", tdtype(dt))
    ref = oracle.update_chain_uneven(n, t, off, A.double().cpu().numpy(), nthreads=8)
    tol = {cj.F64: TOL64, cj.F32: TOL32, cj.BF16: 2e-2}[dt]
    plan = cj.GroupPlan(dt, n, t)
    try:
        plan.wait()
        count = plan.use_dispatcher()
        assert count == {cj.F64: 1, cj.F32: 4, cj.BF16: 3}[dt]
        for v in range(count):
            plan.use_dispatcher(v)
            d = plan.dispatcher()
            assert d["state"] == "ready" and d["blocks_per_sm"] >= 1, (v, d)
            for use_graph in (True, False):
                X = torch.full_like(A, float("nan"))
                plan.launch(A, X, use_graph=use_graph)
                torch.cuda.synchronize()
                Xh = X.double().cpu().numpy()
                assert np.all(np.isfinite(Xh)), (v, use_graph)
                worst = max(relF(Xh[off[k]:off[k] + n[k] * n[k]], ref[off[k]:off[k] + n[k] * n[k]])
                            for k in range(len(n)))
                assert worst <= tol, (v, use_graph, worst)
        with pytest.raises(cj.CJError):
            plan.use_dispatcher(count)
    finally:
        plan.destroy()


def test_generic_plan_has_no_dispatcher():
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 50)
    plan = cj.GroupPlan(cj.F64, n, t, flags=cj.FLAG_GENERIC)
    try:
        assert plan.dispatcher()["state"] == "none"
        assert plan.use_dispatcher() == 0
        with pytest.raises(cj.CJError):
            plan.use_dispatcher(0)
    finally:
        plan.destroy()


@pytest.mark.parametrize("dt", [cj.F64, cj.F32, cj.BF16])
@pytest.mark.parametrize("use_graph", [True, False])
def test_grouped_plan_autotune_keeps_results(dt, use_graph):
    """Plan autotuning: every group's candidates are timed on its own work
    list, the fastest is kept, the graph re-captures (or the streams launch
    the new tiles), results still match."""
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 300)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    ref = oracle.update_chain_uneven(n, t, off, pool)
    plan = cj.GroupPlan(dt, n, t)
    try:
        A = torch.from_numpy(pool).to("cuda", tdtype(dt))
        X = torch.full_like(A, float("nan"))
        changed = plan.autotune(A, X, stream=torch.cuda.current_stream(), max_groups=6, reps=2)
        assert 0 <= changed <= 6
        X.fill_(float("nan"))
        plan.launch(A, X, stream=torch.cuda.current_stream(), use_graph=use_graph)
        torch.cuda.synchronize()
        Xh = X.double().cpu().numpy()
        worst = max(relF(Xh[off[k]:off[k] + n[k] * n[k]], ref[off[k]:off[k] + n[k] * n[k]]) for k in range(len(n)))
        assert worst <= {cj.F64: TOL64, cj.F32: TOL32, cj.BF16: 2e-2}[dt]
    finally:
        plan.destroy()


def test_grouped_handle_direct_launch():
    """One grouped instantiation over a hand-built work list (n = 20)."""
    nn = 20
    steps = np.array([128, 100, 77, 64, 64, 30, 17, 16, 16], dtype=np.int64)
    cnt = len(steps)
    pool = synth.uniform_np(synth.SEED_UNEVEN, 0, cnt * nn * nn)
    ref = np.empty_like(pool)
    for k in range(cnt):
        ref[k * nn * nn:(k + 1) * nn * nn] = oracle.update_chain(
            pool[k * nn * nn:(k + 1) * nn * nn].reshape(1, nn, nn), int(steps[k])).ravel()
    items = np.zeros((cnt, 3), dtype=np.int64)
    items[:, 0] = np.arange(cnt) * nn * nn
    items[:, 1] = steps
    for dt, tile, flags in ((cj.F64, (0, 0, 0, 0), 0), (cj.F64, (0, 0, 0, 0), cj.FLAG_GENERIC),
                            (cj.F32, (5, 2, 0, 0), 0), (cj.F32, (1, 3, 0, 0), 0), (cj.F32, (6, 3, 0, 0), 0),
                            (cj.F32, (8, 2, 0, 0), 0),
                            (cj.BF16, (7, 1, 0, 0), 0), (cj.BF16, (3, 2, 0, 0), 0)):
        h = cj.specialize(cj.K_UPDATE_CHAIN_GROUPED, dt, n=nn, tile=tile, flags=flags)
        it = torch.from_numpy(items).cuda()
        A = torch.from_numpy(pool).to("cuda", tdtype(dt))
        X = torch.full_like(A, float("nan"))
        counter = torch.zeros(1, dtype=torch.int32, device="cuda")
        cj.launch_grouped(h, it, A, X, counter, cnt)
        torch.cuda.synchronize()
        assert relF(X.double().cpu().numpy(), ref) <= {cj.F64: TOL64, cj.F32: TOL32, cj.BF16: 2e-2}[dt], (dt, tile)


# ---------------------------------------------------------------------------
# Full-size launches, checked on seeded samples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,dt", [(3, cj.F64), (32, cj.F64), (12, cj.F32), (32, cj.F32)])
def test_full_size_sweep_sampled(n, dt):
    steps = 64
    batch = synth.chain_batch(n)
    A = synth.chain_inputs_torch(synth.SEED_CHAIN_SWEEP, batch, n, "cuda").to(tdtype(dt))
    X = torch.empty_like(A)
    h = cj.specialize(cj.K_UPDATE_CHAIN, dt, n=n, flags=cj.FLAG_NO_AOT)
    cj.launch_update_chain(h, A, X, steps)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    idx = np.unique(np.concatenate([[0, batch - 1], rng.integers(0, batch, 300)]))
    idx_t = torch.from_numpy(idx).cuda()
    a_s = A[idx_t].double().cpu().numpy()
    if dt == cj.F64:
        np.testing.assert_array_equal(a_s[0], synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, 1, n)[0])
    ref = oracle.update_chain(a_s, steps, nthreads=8)
    assert relF_per_instance(X[idx_t].double().cpu().numpy(), ref) <= (TOL64 if dt == cj.F64 else TOL32)
    del A, X


@pytest.mark.parametrize("dt,lin,lout", [(cj.F64, 0, 3), (cj.F32, 4, 5), (cj.F32, 0, 0), (cj.F32, 1, 2),
                                         (cj.F32, 3, 4)])
def test_full_size_ltimes_sampled(dt, lin, lout):
    """Full size (Z = 2^18) in the bench's launch configuration (the default
    tile: f32 = tensor cores fed by TMA), checked on 400 sampled columns."""
    M, D, G, Z = 36, 96, 32, 1 << 18
    L, _ = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, 1, 1)
    x = synth.uniform_torch(synth.SEED_LTIMES, synth.STREAM_A, D * G * Z, "cuda").view(D, G, Z)
    perm = synth.LAYOUT_PERMS[lin]
    xin = x.permute(*perm).contiguous().to(tdtype(dt)).view(-1)
    Lt = torch.from_numpy(L).to("cuda", tdtype(dt))
    out = torch.empty(M * G * Z, device="cuda", dtype=tdtype(dt))
    h = cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D)
    tma0 = cj.stats()["launches_tma"]
    cj.launch_ltimes(h, Lt, xin, out, G, Z)
    torch.cuda.synchronize()
    assert cj.stats()["launches_tma"] - tma0 == (1 if dt == cj.F32 else 0)
    if dt == cj.F32:
        assert h.wait_timeouts() == 0
    rng = np.random.default_rng(5)
    gs = rng.integers(0, G, 400)
    zs = rng.integers(0, Z, 400)
    cols = x[:, torch.from_numpy(gs).cuda(), torch.from_numpy(zs).cuda()].to(tdtype(dt)).double().cpu().numpy()
    ref = oracle.ltimes(L, cols.ravel(), 1, len(gs), 0, 0).reshape(M, len(gs))
    pout = out.view(*[(M, G, Z)[p] for p in synth.LAYOUT_PERMS[lout]])
    inv = np.argsort(synth.LAYOUT_PERMS[lout])
    canon = pout.permute(*inv)
    got = canon[:, torch.from_numpy(gs).cuda(), torch.from_numpy(zs).cuda()].double().cpu().numpy()
    assert relF(got, ref) <= (TOL64 if dt == cj.F64 else TOL32)
    del x, xin, out


# ---------------------------------------------------------------------------
# LPlusTimes: in += Lp . out
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lin,lout", [(0, 0), (3, 1), (4, 5), (2, 3)])
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
@pytest.mark.parametrize("generic", [False, True])
def test_lplustimes_accumulates(lin, lout, dt, generic):
    M, D, G, Z = 36, 96, 5, 41
    Lp = synth.uniform_np(0xC1A6, 0, D * M).reshape(D, M)
    y = synth.uniform_np(0xC1A7, 0, M * G * Z).reshape(M, G, Z)
    base = synth.uniform_np(0xC1A8, 0, D * G * Z).reshape(D, G, Z)
    ref_phys = oracle.lplustimes(Lp, synth.to_layout(y, lout).ravel(), synth.to_layout(base, lin).ravel(), G, Z,
                                 lin, lout)
    h = cj.specialize(cj.K_LPLUSTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D,
                      flags=cj.FLAG_GENERIC if generic else 0)
    tt = tdtype(dt)
    Lt = torch.from_numpy(Lp).to("cuda", tt)
    yt = torch.from_numpy(synth.to_layout(y, lout).ravel()).to("cuda", tt)
    xt = torch.from_numpy(synth.to_layout(base, lin).ravel()).to("cuda", tt)
    cj.launch_lplustimes(h, Lt, yt, xt, G, Z)
    torch.cuda.synchronize()
    got = xt.double().cpu().numpy()
    assert relF(got, ref_phys) <= (TOL64 if dt == cj.F64 else TOL32)


@pytest.mark.parametrize("lin,lout", [(0, 0), (3, 1), (4, 5), (2, 3), (1, 4)])
@pytest.mark.parametrize("mode5", [False, True])
def test_lplustimes_tcgen05(lin, lout, mode5):
    """LPlusTimes on mode 4 (the swapped problem: 96 output rows, K = 36)."""
    M, D, G, Z = 36, 96, 5, 41
    Lp = synth.uniform_np(0xC1A6, 0, D * M).reshape(D, M)
    y = synth.uniform_np(0xC1A7, 0, M * G * Z).reshape(M, G, Z)
    base = synth.uniform_np(0xC1A8, 0, D * G * Z).reshape(D, G, Z)
    ref_phys = oracle.lplustimes(Lp, synth.to_layout(y, lout).ravel(), synth.to_layout(base, lin).ravel(), G, Z,
                                 lin, lout)
    h = cj.specialize(cj.K_LPLUSTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D,
                      tile=tma_tile(lout, lin, boxes=2, stages=2, nconv=4) if mode5
                      else tc_tile(lout, lin, stages=3, nprod=4))
    Lt = torch.from_numpy(Lp).to("cuda", torch.float32)
    yt = torch.from_numpy(synth.to_layout(y, lout).ravel()).to("cuda", torch.float32)
    xt = torch.from_numpy(synth.to_layout(base, lin).ravel()).to("cuda", torch.float32)
    cj.launch_lplustimes(h, Lt, yt, xt, G, Z)
    torch.cuda.synchronize()
    assert relF(xt.double().cpu().numpy(), ref_phys) <= TOL32
    assert h.wait_timeouts() == 0
