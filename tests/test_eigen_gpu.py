"""The paper's literal Eigen benchmark recurrence on the GPU (Sec. 5,
Listing eigen1): M_{k+1} = Ones + c (M_k + M_k M_k), batched, specialized
(N a template argument) and generic (runtime N), against the FP64 oracle.

With the listing's start M_0(i, j) = i + N j the values grow without bound, so
those comparisons run a few repeats; random starts in [-1, 1) with c = 5e-5
stay near Ones and run longer."""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True)
    yield
    cj.shutdown()


def run(h, M0, repeat, c, dt):
    tt = torch.float64 if dt == cj.F64 else torch.float32
    a = torch.from_numpy(np.ascontiguousarray(M0)).to("cuda", tt)
    out = torch.full_like(a, float("nan"))
    cj.launch_eigen(h, a, out, repeat, c, batch=M0.shape[0])
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def rel_per_instance(x, ref):
    return max(np.linalg.norm(x[b] - ref[b]) / np.linalg.norm(ref[b]) for b in range(ref.shape[0]))


@pytest.mark.parametrize("n", list(range(1, 17)))
@pytest.mark.parametrize("generic", [False, True])
def test_listing_start_f64(n, generic):
    rep = 4
    M0 = np.repeat(oracle.eigen_start(n)[None], 3, axis=0)
    h = cj.specialize(cj.K_EIGEN_RECURRENCE, cj.F64, n=n, flags=cj.FLAG_GENERIC if generic else 0)
    assert h.variant == ("generic" if generic else "jit")
    got = run(h, M0, rep, 5e-5, cj.F64)
    ref = np.repeat(oracle.eigen_bench(n, rep)[None], 3, axis=0)
    assert np.all(np.isfinite(ref))
    assert rel_per_instance(got, ref) <= TOL64


@pytest.mark.parametrize("n,tile", [(3, None), (8, (1, 5, 0, 0)), (13, None), (16, (1, 2, 0, 0)), (32, None)])
@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
def test_random_starts(n, tile, dt):
    rep, c = 40, 5e-5
    batch = 301                                    # ragged against every tile
    M0 = synth.uniform_np(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, batch * n * n).reshape(batch, n, n)
    ref = oracle.eigen_recurrence(M0, rep, c)
    kw = {} if tile is None else {"tile": tile}
    h = cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, **kw)
    g = cj.specialize(cj.K_EIGEN_RECURRENCE, dt, n=n, flags=cj.FLAG_GENERIC)
    tol = TOL64 if dt == cj.F64 else TOL32
    assert rel_per_instance(run(h, M0, rep, c, dt), ref) <= tol
    assert rel_per_instance(run(g, M0, rep, c, dt), ref) <= tol


def test_zero_repeats_copy_the_start():
    n = 6
    M0 = synth.uniform_np(3, 0, 10 * n * n).reshape(10, n, n)
    h = cj.specialize(cj.K_EIGEN_RECURRENCE, cj.F64, n=n)
    np.testing.assert_array_equal(run(h, M0, 0, 5e-5, cj.F64), M0)


@pytest.mark.parametrize("n,ipb", [(1, 3), (2, 128), (5, 7), (8, 32), (9, 25), (13, 18), (16, 16), (17, 14),
                                   (24, 10), (31, 8), (32, 8)])
def test_two_rows_per_thread_f32(n, ipb):
    """Tile mapping 2 (two rows of M per thread, FP32) against the FP64
    oracle, on a batch ragged against the tile, and bit for bit against the
    one-row kernel: per element both do the same operations in the same order."""
    rep, c = 40, 5e-5
    batch = 301
    M0 = synth.uniform_np(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, batch * n * n).reshape(batch, n, n)
    ref = oracle.eigen_recurrence(M0, rep, c)
    h2 = cj.specialize(cj.K_EIGEN_RECURRENCE, cj.F32, n=n, tile=(2, ipb, 0, 0))
    h1 = cj.specialize(cj.K_EIGEN_RECURRENCE, cj.F32, n=n, tile=(1, max(1, 128 // n), 0, 0))
    got2 = run(h2, M0, rep, c, cj.F32)
    assert rel_per_instance(got2, ref) <= TOL32
    np.testing.assert_array_equal(got2, run(h1, M0, rep, c, cj.F32))
