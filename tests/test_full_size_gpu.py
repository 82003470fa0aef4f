"""GPU parity at the workloads' own sizes, element by element against the oracle.

* LTimes, every one of the 36 (in, out) storage-order pairs at M = 36, D = 96,
  G = 32, Z = 2^12 (131,072 columns: the persistent kernels run many tiles per
  block), in FP64 (FMA-pipe default tile) and FP32 (tcgen05 + TMA default
  tile): relative Frobenius error over the whole output and per m-slice.  The
  oracle is evaluated once, in the canonical orders; its six-orders pin shows
  the other orders give the same values bit for bit.
* The uneven batch at its full size, 10,000 instances (N log-uniform in
  [2, 64], T uniform in [16, 128]), through the grouped plan in FP64, FP32 and
  BF16 -- its one-launch dispatcher and its per-group kernels, each as a graph
  and directly -- every instance checked against the oracle.  BF16 runs N >= 16 on
  bf16 tensor-core operands with FP32 state and N < 16 in FP32.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32, TOLBF16 = 1e-12, 1e-5, 2e-2
M, D, G, Z = 36, 96, 32, 1 << 12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True, compile_threads=4)
    yield
    cj.shutdown()


@pytest.fixture(scope="module")
def lt_full():
    L, _ = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, 1, 1)
    x = synth.uniform_np(synth.SEED_LTIMES, synth.STREAM_A, D * G * Z).reshape(D, G, Z)
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0, nthreads=16).reshape(M, G, Z)
    return L, torch.from_numpy(x).cuda(), ref


def relF(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def canonical(out, lout):
    """Physical out buffer in order lout -> logical [m][g][z] (on the GPU)."""
    pout = out.view(*[(M, G, Z)[p] for p in synth.LAYOUT_PERMS[lout]])
    return pout.permute(*np.argsort(synth.LAYOUT_PERMS[lout]).tolist())


@pytest.mark.parametrize("dt", [cj.F64, cj.F32])
@pytest.mark.parametrize("lin", range(6))
@pytest.mark.parametrize("lout", range(6))
def test_ltimes_all_orders_z4096(lt_full, dt, lin, lout):
    L, x, ref = lt_full
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    tol = TOL64 if dt == cj.F64 else TOL32
    xin = x.permute(*synth.LAYOUT_PERMS[lin]).contiguous().view(-1).to(tdt)
    out = torch.full((M * G * Z,), float("nan"), device="cuda", dtype=tdt)
    h = cj.specialize(cj.K_LTIMES, dt, layout_a=lin, layout_b=lout, m=M, d=D)
    assert h.variant == "jit"
    cj.launch_ltimes(h, torch.from_numpy(L).to("cuda", tdt), xin, out, G, Z)
    torch.cuda.synchronize()
    if dt == cj.F32:
        assert h.wait_timeouts() == 0
    got = canonical(out, lout).double().cpu().numpy()
    assert np.all(np.isfinite(got))
    assert relF(got, ref) <= tol
    per_m = [relF(got[m], ref[m]) for m in range(M)]
    assert max(per_m) <= tol, int(np.argmax(per_m))


@pytest.fixture(scope="module")
def uneven_full():
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 10000)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    ref64 = oracle.update_chain_uneven(n, t, off, pool, nthreads=16)
    # FP32 and BF16 plans read the pool rounded to FP32: their reference
    # starts from the same rounded inputs
    ref32 = oracle.update_chain_uneven(n, t, off, pool.astype(np.float32).astype(np.float64), nthreads=16)
    return n, t, pool, off, ref64, ref32


def per_instance_relF(got, ref, n, off):
    errs = np.empty(len(n))
    for nn in np.unique(n):
        idx = np.nonzero(n == nn)[0]
        rows = off[idx][:, None] + np.arange(nn * nn)[None, :]
        errs[idx] = np.linalg.norm(got[rows] - ref[rows], axis=1) / np.linalg.norm(ref[rows], axis=1)
    return errs


@pytest.mark.parametrize("dt", [cj.F64, cj.F32, cj.BF16])
def test_uneven_batch_10000_every_instance(uneven_full, dt):
    n, t, pool, off, ref64, ref32 = uneven_full
    tdt = torch.float64 if dt == cj.F64 else torch.float32
    ref = ref64 if dt == cj.F64 else ref32
    plan = cj.GroupPlan(dt, n, t)
    try:
        A = torch.from_numpy(pool).to("cuda", tdt)
        plan.wait()
        assert plan.dispatcher()["state"] == "ready"
        for use_graph, per_group in ((True, False), (False, False), (True, True), (False, True)):
            X = torch.full_like(A, float("nan"))
            plan.launch(A, X, use_graph=use_graph, per_group=per_group)
            torch.cuda.synchronize()
            got = X.double().cpu().numpy()
            assert np.all(np.isfinite(got)), (use_graph, per_group)
            err = per_instance_relF(got, ref, n, off)
            if dt == cj.F64:
                assert err.max() <= TOL64, (use_graph, per_group, err.max())
            elif dt == cj.F32:
                assert err.max() <= TOL32, (use_graph, per_group, err.max())
            else:
                big = n >= 16
                assert err[big].max() <= TOLBF16, (use_graph, per_group, err[big].max())
                assert err[~big].max() <= TOL32, (use_graph, per_group, err[~big].max())
    finally:
        plan.destroy()
