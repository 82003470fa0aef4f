"""The learned cost model end to end on the GPU: autotuner timings -> MLP
trained with libcj's own kernels -> choices on held-out requests.

A reduced version of the full procedure (bench.py --workload costmodel):
fewer training sizes and 150 held-out requests.  The trained network must
choose clearly better tiles than a uniformly random candidate; its regret
and the default tile's ("no model") are printed."""
import math

import numpy as np
import pytest

from paper_1904_08555_b300 import cj, costmodel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    cj.init(sync=False, compile_threads=os.cpu_count() or 4)
    yield
    cj.shutdown()


def test_trained_model_beats_random_choice():
    train = [r for r in costmodel.training_requests()
             if r.kernel == cj.K_LTIMES or r[2] in (3, 5, 8, 12, 16, 24, 32, 48, 64)]
    held = costmodel.heldout_requests(150)
    timer = costmodel.Timer(reps=3)
    timer.prefetch(train + held)
    X, y, _ = costmodel.dataset(timer, train)
    assert len(y) > 200 and np.all(np.isfinite(y))
    model = costmodel.CostModel()
    try:
        final = model.fit(X, y, steps=2500)
        assert final < 0.2           # standardised targets: most variance explained
        reg = costmodel.evaluate(model, timer, held)
    finally:
        model.destroy()
    s = costmodel.summarize(reg)
    print("regret", {k: {m: round(v, 4) for m, v in d.items()} for k, d in s.items()})
    assert s["model"]["geomean"] < s["random"]["geomean"]
    assert s["model"]["geomean"] < 0.25
    assert all(math.isfinite(v) for v in reg["model"])
