"""The learned cost model end to end on the GPU: autotuner timings -> MLP
trained with libcj's own kernels -> choices on unseen requests.

A reduced version of the full procedure (bench.py --workload costmodel): the
full training set and 150 held-out requests, none of which is a training
request (other chain sizes, other LTimes storage-order pairs).  On those
unseen requests the trained network must choose better tiles than the
library's default rule ("no model") and than a uniformly random candidate,
measured as geometric-mean regret against exhaustive autotuning."""
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
    cj.init(sync=False, compile_threads=min(16, os.cpu_count() or 4))
    yield
    cj.shutdown()


def test_trained_model_beats_the_default_rule_on_unseen_requests():
    train = costmodel.training_requests()
    held = costmodel.heldout_requests(150)
    assert not set(train) & set(held)
    timer = costmodel.Timer(reps=3)
    timer.prefetch(train + held)
    X, y, _ = costmodel.dataset(timer, train)
    assert len(y) > 500 and np.all(np.isfinite(y))
    model = costmodel.CostModel()
    try:
        model.fit(X, y, steps=4000)
        rmse = float(np.sqrt(np.mean((model.predict(X) - y) ** 2)))
        assert rmse < 0.25           # log-ms fit on the training table
        reg = costmodel.evaluate(model, timer, held)
    finally:
        model.destroy()
    s = costmodel.summarize(reg)
    print("unseen regret", {k: {m: round(v, 4) for m, v in d.items()} for k, d in s.items()})
    assert all(math.isfinite(v) for v in reg["model"])
    assert s["model"]["geomean"] < s["default"]["geomean"]
    assert s["model"]["geomean"] < s["random"]["geomean"]
    assert s["model"]["geomean"] < 0.10
