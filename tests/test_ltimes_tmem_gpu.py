"""LTimes and LPlusTimes on tcgen05 with the A operand in tensor memory (tile
mode 6) against the FP64 oracle.

Mode 6 is mode 5 (TMA boxes of `in`, converter warps, 3xTF32 on
tcgen05.mma with TMEM accumulators) with the converters writing the tf32
hi/lo operand straight into tensor memory (tcgen05.st) and the MMAs reading A
from there.  Each converter warp owns the tile rows of its TMEM lane quarter,
so the cases below cover every storage-order pair, both converter counts (4:
one warp per quarter takes all 32 directions of a box; 8: two warps take 16
each), TMEM stage rings up to the 512-column limit, ragged tiles and K blocks,
the mode-4 twin where `in` admits no tensor map, the accumulating epilogue of
LPlusTimes, and the bounded waits."""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True, compile_threads=2)
    yield
    cj.shutdown()


def box_tg(lin, lout):
    """g extent of the 128-column tile: the library's box-shape rule (8 x 16 where
    in and out have different fastest column axes)."""
    gi, go = lin in (1, 4), lout in (1, 4)
    zi, zo = lin in (0, 2), lout in (0, 2)
    if not (gi or go):
        return 1
    return 8 if (gi and zo) or (go and zi) else 32


def tmem_tile(lin, lout, boxes=4, stages=2, nconv=8, tg=None):
    """Mode 6: `boxes` TMA boxes, `stages` TMEM operand stages, `nconv` converter warps."""
    tg = box_tg(lin, lout) if tg is None else tg
    return (tg, 128 // tg, 32 * (6 + nconv), (boxes << 20) | (6 << 16) | (stages << 8) | nconv)


def run_ltimes(h, L, x_canon, lin, lout):
    M, D = L.shape
    _, G, Z = x_canon.shape
    Lt = torch.from_numpy(L).to("cuda", torch.float32)
    xt = torch.from_numpy(synth.to_layout(x_canon, lin).ravel()).to("cuda", torch.float32)
    out = torch.full((M * G * Z,), float("nan"), device="cuda", dtype=torch.float32)
    cj.launch_ltimes(h, Lt, xt, out, G, Z)
    torch.cuda.synchronize()
    return synth.from_layout(out.cpu().numpy(), lout, (M, G, Z)).astype(np.float64)


def relF(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def check(M, D, G, Z, lin, lout, tile, tma=True, nthreads=4):
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=nthreads).reshape(M, G, Z)
    h = cj.specialize(cj.K_LTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D, tile=tile)
    assert h.variant == "jit"
    before = cj.stats()
    got = run_ltimes(h, L, x, lin, lout)
    after = cj.stats()
    assert not np.isnan(got).any()
    # every column and moment, and each m-slice on its own
    assert relF(got, ref) <= TOL32
    for m in range(M):
        assert np.linalg.norm(got[m] - ref[m]) <= TOL32 * max(np.linalg.norm(ref[m]), 1e-30)
    assert after["launches_tma"] - before["launches_tma"] == (1 if tma else 0)
    assert after["launches_tma_fallback"] - before["launches_tma_fallback"] == (0 if tma else 1)
    assert h.wait_timeouts() == 0


@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
def test_every_order_pair(lin, lout):
    """G and Z multiples of 4 (a tensor map for every order of `in`), Z ragged against every box."""
    check(36, 96, 8, 200, lin, lout, tmem_tile(lin, lout))


@pytest.mark.parametrize("lin,lout,boxes,stages,nconv", [
    (0, 0, 6, 4, 8), (1, 4, 4, 2, 4), (3, 5, 8, 6, 8), (4, 0, 2, 3, 4), (5, 3, 6, 4, 4), (2, 1, 3, 5, 8),
])
def test_rings_and_converter_counts(lin, lout, boxes, stages, nconv):
    """TMA rings of 2-8 boxes, TMEM rings of 2-6 stages (M = 36: 128 + 6 x 64 = 512 columns)."""
    check(36, 96, 8, 200, lin, lout, tmem_tile(lin, lout, boxes, stages, nconv))


@pytest.mark.parametrize("lin,lout,tg", [(0, 0, None), (3, 5, None), (4, 1, None), (1, 4, 8), (2, 3, 1), (5, 0, 8),
                                         (1, 0, None), (4, 2, 16)])
def test_many_tiles_per_block(lin, lout, tg):
    """2,048 tiles over at most one block per SM: the persistent loop wraps both rings many times."""
    check(36, 96, 32, 8192, lin, lout, tmem_tile(lin, lout, boxes=6, stages=4, tg=tg), nthreads=8)


@pytest.mark.parametrize("M,D,G,Z,lin,lout,boxes,stages,nconv", [
    (37, 12, 4, 52, 0, 0, 4, 2, 8),      # one K block, directions 12..31 from TMA zero fill
    (9, 8, 4, 36, 1, 4, 2, 2, 4),        # g innermost, 32-wide g box
    (4, 100, 4, 300, 2, 3, 3, 3, 4),     # four K blocks, ragged; m-fastest out
    (64, 128, 3, 70, 3, 3, 2, 2, 8),     # d innermost (128-byte swizzle), ragged G and Z
    (16, 40, 12, 24, 5, 2, 2, 4, 8),     # d innermost, D not a multiple of 32
    (64, 64, 4, 96, 2, 0, 4, 6, 8),      # NP = 64: two 64-column accumulators + 6 stages = 512 columns
    (50, 33, 8, 64, 4, 5, 4, 3, 4),      # NP = 64 with 14 padded moments, D just past one K block
])
def test_shapes(M, D, G, Z, lin, lout, boxes, stages, nconv):
    check(M, D, G, Z, lin, lout, tmem_tile(lin, lout, boxes, stages, nconv))


@pytest.mark.parametrize("lin,lout", [(0, 0), (1, 4), (4, 2), (3, 3), (5, 1), (2, 5)])
def test_twin_without_tensor_map(lin, lout):
    """G = 5, Z = 37 admit no tensor map when g or z is innermost: the launch runs
    the mode-4 twin compiled into the same module; d innermost (D = 96) stays on TMA."""
    check(36, 96, 5, 37, lin, lout, tmem_tile(lin, lout), tma=lin in (3, 5))


def test_tiles_beyond_tensor_memory_are_rejected():
    """M = 64 (two 64-column accumulators) leaves room for 6 stages of 64 columns, not 7."""
    with pytest.raises(cj.CJError):
        cj.specialize(cj.K_LTIMES, cj.F32, m=64, d=64, tile=tmem_tile(0, 0, 4, 7, 8))
    with pytest.raises(cj.CJError):   # converter warps come in whole lane quarters
        cj.specialize(cj.K_LTIMES, cj.F32, m=36, d=96, tile=tmem_tile(0, 0, 4, 2, 2))


@pytest.mark.parametrize("lin,lout", [(0, 0), (3, 1), (4, 5), (2, 3), (1, 4)])
def test_lplustimes(lin, lout):
    """LPlusTimes on mode 6: the swapped problem (96 output rows: NP = 96, 5 stages
    fit TMEM) with the accumulating epilogue."""
    M, D, G, Z = 36, 96, 8, 44
    Lp = synth.uniform_np(0xC1A6, 0, D * M).reshape(D, M)
    y = synth.uniform_np(0xC1A7, 0, M * G * Z).reshape(M, G, Z)
    base = synth.uniform_np(0xC1A8, 0, D * G * Z).reshape(D, G, Z)
    ref_phys = oracle.lplustimes(Lp, synth.to_layout(y, lout).ravel(), synth.to_layout(base, lin).ravel(), G, Z,
                                 lin, lout)
    h = cj.specialize(cj.K_LPLUSTIMES, cj.F32, layout_a=lin, layout_b=lout, m=M, d=D,
                      tile=tmem_tile(lout, lin, boxes=4, stages=5, nconv=4))
    Lt = torch.from_numpy(Lp).to("cuda", torch.float32)
    yt = torch.from_numpy(synth.to_layout(y, lout).ravel()).to("cuda", torch.float32)
    xt = torch.from_numpy(synth.to_layout(base, lin).ravel()).to("cuda", torch.float32)
    cj.launch_lplustimes(h, Lt, yt, xt, G, Z)
    torch.cuda.synchronize()
    assert relF(xt.double().cpu().numpy(), ref_phys) <= TOL32
    assert h.wait_timeouts() == 0
