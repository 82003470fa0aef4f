"""Asynchronous specialization on the GPU: a miss launches the generic
kernel at once, the background thread swaps in the JIT kernel, and results
match the oracle before and after the swap (and after a failed compile)."""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=False, compile_threads=1)
    yield
    cj.shutdown()


def relF_max(x, ref, n):
    x = x.reshape(-1, n * n)
    ref = ref.reshape(-1, n * n)
    return float(np.max(np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def test_generic_first_then_jit():
    n, steps, batch = 9, 50, 333
    A_np = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    ref = oracle.update_chain(A_np, steps)
    A = torch.from_numpy(A_np).cuda()
    before = cj.stats()
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, tile=(1, 14, 0, 0))
    assert h.variant == "generic"          # the compile takes far longer than this
    X = torch.empty_like(A)
    cj.launch_update_chain(h, A, X, steps)
    torch.cuda.synchronize()
    assert relF_max(X.cpu().numpy(), ref, n) <= 1e-12
    assert h.wait(-1) == cj.CJ_OK
    assert h.variant == "jit"
    X2 = torch.empty_like(A)
    cj.launch_update_chain(h, A, X2, steps)
    torch.cuda.synchronize()
    assert relF_max(X2.cpu().numpy(), ref, n) <= 1e-12
    after = cj.stats()
    assert after["launches_generic"] - before["launches_generic"] == 1
    assert after["launches_jit"] - before["launches_jit"] == 1


def test_failed_compile_keeps_generic_results_correct():
    n, steps, batch = 6, 20, 100
    A_np = synth.chain_inputs_np(synth.SEED_CHAIN_SWEEP, batch, n)
    ref = oracle.update_chain(A_np, steps)
    h = cj.specialize(cj.K_UPDATE_CHAIN, cj.F64, n=n, flags=cj.FLAG_INJECT_COMPILE_ERROR)
    assert h.wait(-1) == cj.CJ_ERR_COMPILE
    assert h.variant == "generic"
    A = torch.from_numpy(A_np).cuda()
    X = torch.empty_like(A)
    cj.launch_update_chain(h, A, X, steps)
    torch.cuda.synchronize()
    assert relF_max(X.cpu().numpy(), ref, n) <= 1e-12


def test_grouped_plan_recaptures_after_upgrade():
    n, t = synth.uneven_sizes(synth.SEED_UNEVEN + 1, 150)
    pool, off = synth.uneven_inputs_np(synth.SEED_UNEVEN + 1, n)
    ref = oracle.update_chain_uneven(n, t, off, pool)
    plan = cj.GroupPlan(cj.F64, n, t)
    try:
        A = torch.from_numpy(pool).cuda()
        s = torch.cuda.Stream()
        for phase in range(2):
            X = torch.full_like(A, float("nan"))
            with torch.cuda.stream(s):
                plan.launch(A, X, stream=s, use_graph=True)
            s.synchronize()
            Xh = X.cpu().numpy()
            for k in range(len(n)):
                sl = slice(off[k], off[k] + n[k] * n[k])
                assert np.linalg.norm(Xh[sl] - ref[sl]) <= 1e-12 * np.linalg.norm(ref[sl])
            if phase == 0:
                # let every group's specialization finish; the next launch re-captures
                for nn in np.unique(n):
                    h = cj.specialize(cj.K_UPDATE_CHAIN_GROUPED, cj.F64, n=int(nn))
                    assert h.wait(-1) == cj.CJ_OK
    finally:
        plan.destroy()
