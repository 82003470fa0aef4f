"""Failure detection of the tensor-core LTimes kernels without a GPU fault.

Every barrier wait in the tcgen05 kernels (tile modes 4-6) is bounded:
after about a second a block raises its abort flag, waits for its own
tensor-core work and TMA copies, frees its tensor memory, counts the event
and returns.  CJ_FLAG_INJECT_WAIT_TIMEOUT compiles the kernel with
producers that never signal a filled stage (a barrier that nothing
completes), so every block's wait runs out; the host reads the count, and the
context stays usable for a correct launch afterwards."""
import numpy as np
import pytest

import oracle
import synth
from paper_1904_08555_b300 import cj

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.injects_wait_timeouts]

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cj.init(sync=True)
    yield
    cj.shutdown()


@pytest.mark.parametrize("tile", [
    (1, 128, 32 * 14, (2 << 20) | (5 << 16) | (2 << 8) | 8),   # mode 5: TMA boxes in flight at the stop
    (1, 128, 32 * 14, (2 << 20) | (6 << 16) | (2 << 8) | 8),   # mode 6: operands in tensor memory
    (1, 128, 32 * 13, (4 << 16) | (2 << 8) | 8),               # mode 4: register producers
])
def test_expired_waits_are_reported_and_the_context_survives(tile):
    M, D, G, Z = 36, 96, 8, 256          # 16 tiles: 16 blocks, each waits once and stops
    L, x = synth.ltimes_inputs_np(synth.SEED_LTIMES, M, D, G, Z)
    Lt = torch.from_numpy(L).to("cuda", torch.float32)
    xt = torch.from_numpy(x.ravel()).to("cuda", torch.float32)
    out = torch.zeros(M * G * Z, device="cuda", dtype=torch.float32)
    bad = cj.specialize(cj.K_LTIMES, cj.F32, m=M, d=D, tile=tile, flags=cj.FLAG_INJECT_WAIT_TIMEOUT)
    assert bad.wait_timeouts(reset=True) == 0
    cj.launch_ltimes(bad, Lt, xt, out, G, Z)
    torch.cuda.synchronize()                    # returns: no block waits forever
    assert cj.stats()["wait_timeouts"] >= 1    # surfaced in the library-wide counters
    n = bad.wait_timeouts(reset=True)
    assert 1 <= n <= 16, n
    assert bad.wait_timeouts() == 0             # reset
    good = cj.specialize(cj.K_LTIMES, cj.F32, m=M, d=D, tile=tile)
    cj.launch_ltimes(good, Lt, xt, out, G, Z)
    torch.cuda.synchronize()
    ref = oracle.ltimes(L, x.ravel(), G, Z, 0, 0).reshape(M, G, Z)
    got = out.double().cpu().numpy().reshape(M, G, Z)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL32
    assert good.wait_timeouts() == 0
    assert cj.stats()["wait_timeouts"] == 0     # the total over all modules, after the reset
