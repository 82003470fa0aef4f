"""The allocation-free uneven update chain (cj_update_chain_uneven_noalloc).

Callers that must not allocate device memory -- code under a device-memory
budget owned by another allocator, or on a latency-critical path where
cudaMalloc/cudaFree may synchronize the device -- use this entry point; it
keeps its scratch (work list and counters) in a fixed array inside the
library.  These tests call it through the C ABI and compare its output with
the FP64 oracle directly and with the existing grouped plan's
(cj_group_plan_*), twice in a row, at the same tolerances as the other parity
tests (FP64 1e-12, FP32 1e-5 relative Frobenius error per instance).  One
call runs while the library is not initialised (the entry point does not need
cj_init); the others initialise and shut the library down themselves, so the
module passes alone in a fresh process or after other tests.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
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


def sizes_with_ends(seed, count):
    """An uneven draw whose first instances are n = 1 and n = 64 (the ends of
    the supported range)."""
    n, t = synth.uneven_sizes(seed, count)
    n[0], t[0] = 1, 37
    n[1], t[1] = 64, 128
    return n, t


def test_noalloc_without_init_matches_oracle():
    """Runs first in this module, while the library is shut down."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.shutdown()                       # no-op unless an earlier module left it initialised
    with pytest.raises(cj.CJError):
        cj.stats()                      # the library is not initialised here
    n, t = sizes_with_ends(synth.SEED_UNEVEN + 3, 120)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN + 3, n)
    ref = oracle.update_chain_uneven(n, t, off, pool)
    A = torch.from_numpy(pool).cuda()
    X = torch.full_like(A, float("nan"))
    cj.update_chain_uneven_noalloc(cj.F64, n, t, A, X)
    torch.cuda.synchronize()
    assert per_instance_relF(X.cpu().numpy(), ref, n, off) <= 1e-12


@pytest.mark.parametrize("dtype,tol", [(cj.F64, 1e-12), (cj.F32, 1e-5)])
def test_noalloc_matches_oracle_and_grouped_plan_on_two_calls(lib, dtype, tol):
    tdt = torch.float64 if dtype == cj.F64 else torch.float32
    n, t = sizes_with_ends(synth.SEED_UNEVEN, 700)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN, n)
    A = torch.from_numpy(pool).to("cuda", tdt)
    ref = oracle.update_chain_uneven(n, t, off, A.double().cpu().numpy())

    plan = cj.GroupPlan(dtype, n, t)
    try:
        X_plan = torch.full_like(A, float("nan"))
        plan.launch(A, X_plan, use_graph=False)
        torch.cuda.synchronize()
        plan_out = X_plan.double().cpu().numpy()
    finally:
        plan.destroy()
    assert per_instance_relF(plan_out, ref, n, off) <= tol

    for call in range(2):
        X = torch.full_like(A, float("nan"))
        cj.update_chain_uneven_noalloc(dtype, n, t, A, X)
        torch.cuda.synchronize()
        got = X.double().cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert per_instance_relF(got, ref, n, off) <= tol, call
        assert per_instance_relF(got, plan_out, n, off) <= 2 * tol, call


def test_noalloc_second_call_with_other_sizes(lib):
    """The scratch keeps the previous call's contents; a different, smaller
    batch right after a larger one must still be exact."""
    for seed, count in ((synth.SEED_UNEVEN + 7, 300), (synth.SEED_UNEVEN + 8, 40)):
        n, t = synth.uneven_sizes(seed, count)
        pool, off = synth.uneven_inputs_np(seed, n)
        ref = oracle.update_chain_uneven(n, t, off, pool)
        A = torch.from_numpy(pool).cuda()
        X = torch.empty_like(A)
        cj.update_chain_uneven_noalloc(cj.F64, n, t, A, X)
        torch.cuda.synchronize()
        assert per_instance_relF(X.cpu().numpy(), ref, n, off) <= 1e-12


def test_noalloc_at_its_instance_limit(lib):
    """count == CJ_NOALLOC_MAX_INSTANCES fills the whole work list."""
    count = cj.NOALLOC_MAX_INSTANCES
    rng_n, rng_t = synth.uneven_sizes(synth.SEED_UNEVEN + 9, count, n_lo=1, n_hi=3, t_lo=1, t_hi=20)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN + 9, rng_n)
    ref = oracle.update_chain_uneven(rng_n, rng_t, off, pool)
    A = torch.from_numpy(pool).cuda()
    X = torch.full_like(A, float("nan"))
    cj.update_chain_uneven_noalloc(cj.F64, rng_n, rng_t, A, X)
    torch.cuda.synchronize()
    got = X.cpu().numpy()
    assert np.all(np.isfinite(got))
    # every instance, vectorised per size: rel-F per instance
    for nn in np.unique(rng_n):
        idx = np.nonzero(rng_n == nn)[0]
        rows = off[idx][:, None] + np.arange(nn * nn)[None, :]
        err = np.linalg.norm(got[rows] - ref[rows], axis=1) / np.linalg.norm(ref[rows], axis=1)
        assert err.max() <= 1e-12, (nn, err.max())


def test_noalloc_rejects_more_instances_than_its_scratch_holds(lib):
    count = cj.NOALLOC_MAX_INSTANCES + 1
    n = np.full(count, 2, dtype=np.int32)
    t = np.full(count, 16, dtype=np.int32)
    A = torch.zeros(count * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(cj.CJError) as e:
        cj.update_chain_uneven_noalloc(cj.F64, n, t, A, A)
    assert e.value.status == cj.CJ_ERR_INVALID_ARG
    assert "scratch limit" in cj.last_error()


def test_binding_rejects_a_pool_of_the_wrong_type_or_size(lib):
    """The binding checks the pools before calling into the library."""
    n = np.array([3, 5], dtype=np.int32)
    t = np.array([16, 16], dtype=np.int32)
    short = torch.zeros(9 + 24, dtype=torch.float64, device="cuda")
    wrong = torch.zeros(9 + 25, dtype=torch.float32, device="cuda")
    for bad in (short, wrong):
        with pytest.raises(cj.CJError) as e:
            cj.update_chain_uneven_noalloc(cj.F64, n, t, bad, bad)
        assert e.value.status == cj.CJ_ERR_INVALID_ARG
