"""The allocation-free uneven update chain (cj_update_chain_uneven_noalloc).

Callers that must not allocate device memory -- code under a device-memory
budget owned by another allocator, or on a latency-critical path where
cudaMalloc/cudaFree may synchronize the device -- use this entry point; it
keeps its scratch (work list and counters) in a fixed array inside the
library.  These tests call it through the C ABI twice in a row and compare
its output with the existing grouped plan's (cj_group_plan_*), at the same
tolerances as the other parity tests (FP64 1e-12, FP32 1e-5 relative
Frobenius error per instance).  The module initialises and shuts down the
library itself, so it passes alone in a fresh process or after other tests.
"""
import numpy as np
import pytest

import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True)
    yield
    cj.shutdown()


def per_instance_relF(x, ref, n, off):
    worst = 0.0
    for k in range(len(n)):
        sl = slice(off[k], off[k] + n[k] * n[k])
        worst = max(worst, float(np.linalg.norm(x[sl] - ref[sl]) / np.linalg.norm(ref[sl])))
    return worst


@pytest.mark.parametrize("dtype,tol", [(cj.F64, 1e-12), (cj.F32, 1e-5)])
def test_noalloc_matches_grouped_plan_on_two_calls(dtype, tol):
    tdt = torch.float64 if dtype == cj.F64 else torch.float32
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN, 700)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    A = torch.from_numpy(pool).to("cuda", tdt)

    plan = cj.GroupPlan(dtype, n, t)
    try:
        X_ref = torch.full_like(A, float("nan"))
        plan.launch(A, X_ref, use_graph=False)
        torch.cuda.synchronize()
        ref = X_ref.double().cpu().numpy()
    finally:
        plan.destroy()

    for call in range(2):
        X = torch.full_like(A, float("nan"))
        cj.update_chain_uneven_noalloc(dtype, n, t, A, X)
        torch.cuda.synchronize()
        got = X.double().cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert per_instance_relF(got, ref, n, off) <= tol, call


def test_noalloc_second_call_with_other_sizes():
    """The scratch keeps the previous call's contents; a different, smaller
    batch right after a larger one must still be exact."""
    for seed, count in ((synth.SEED_UNEVEN + 7, 300), (synth.SEED_UNEVEN + 8, 40)):
        n, t = synth.uneven_sizes(seed, count)
        pool, off = synth.uneven_inputs_np(seed, n)
        A = torch.from_numpy(pool).cuda()
        plan = cj.GroupPlan(cj.F64, n, t)
        try:
            X_ref = torch.empty_like(A)
            plan.launch(A, X_ref, use_graph=False)
            X = torch.empty_like(A)
            cj.update_chain_uneven_noalloc(cj.F64, n, t, A, X)
            torch.cuda.synchronize()
            assert per_instance_relF(X.cpu().numpy(), X_ref.cpu().numpy(), n, off) <= 1e-12
        finally:
            plan.destroy()


def test_noalloc_rejects_more_instances_than_its_scratch_holds():
    count = cj.NOALLOC_MAX_INSTANCES + 1
    n = np.full(count, 2, dtype=np.int32)
    t = np.full(count, 16, dtype=np.int32)
    A = torch.zeros(count * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(cj.CJError) as e:
        cj.update_chain_uneven_noalloc(cj.F64, n, t, A, A)
    assert e.value.status == cj.CJ_ERR_INVALID_ARG
    assert "scratch limit" in cj.last_error()
