"""Host logic of the cost-model harness, on the CPU: the seeded held-out
request stream, request marshalling and the regret summary."""
import math

import numpy as np

from paper_1904_08555_b300 import cj, costmodel


def test_heldout_stream_is_seeded_and_in_range():
    a = costmodel.heldout_requests(2000)
    assert a == costmodel.heldout_requests(2000)
    assert a != costmodel.heldout_requests(2000, seed=12345)
    chains = [r for r in a if r.kernel == cj.K_UPDATE_CHAIN]
    lt = [r for r in a if r.kernel == cj.K_LTIMES]
    assert len(chains) + len(lt) == 2000
    # 50/50 kernels and dtypes: binomial(2000, 1/2) has sd 22.4; 5 sd either side
    assert abs(len(chains) - 1000) < 112
    assert abs(sum(r[1] == cj.F64 for r in a) - 1000) < 112
    assert {r[1] for r in a} == {cj.F64, cj.F32}
    assert min(r[2] for r in chains) == 2 and max(r[2] for r in chains) == 64
    assert {r[3] for r in chains} == {0, 1} and all(r[4] == 0 for r in chains)
    assert {r[3] for r in lt} == set(range(6)) and {r[4] for r in lt} == set(range(6))
    assert all(r[2] == 0 for r in lt)


def test_training_requests_cover_every_order_pair_and_size():
    t = costmodel.training_requests()
    assert len(t) == 2 * (len(costmodel.TRAIN_CHAIN_N) * 2 + 36)
    assert len(set(t)) == len(t)
    for dt in (cj.F64, cj.F32):
        assert {(r[3], r[4]) for r in t if r.kernel == cj.K_LTIMES and r[1] == dt} == \
            {(i, o) for i in range(6) for o in range(6)}


def test_request_marshalling():
    r = costmodel.Request((cj.K_LTIMES, cj.F32, 0, 3, 5))
    assert r.kw() == dict(dtype=cj.F32, layout_a=3, layout_b=5, m=36, d=96)
    assert r.batch() == costmodel.LT_G * costmodel.LT_Z
    c = costmodel.Request((cj.K_UPDATE_CHAIN, cj.F64, 12, 1, 0))
    assert c.kw() == dict(dtype=cj.F64, n=12, layout_a=1)
    assert c.batch() == (1 << 22) // 144
    assert costmodel.chain_batch(4096) == 1


def test_summary_statistics():
    # regrets 0 and 0.21: geometric mean of the time ratios 1 and 1.21 is 1.1
    s = costmodel.summarize({"m": np.array([0.0, 0.21]), "z": np.zeros(4)})
    assert math.isclose(s["m"]["geomean"], 0.1, rel_tol=1e-12)
    assert math.isclose(s["m"]["p50"], 0.105, rel_tol=1e-12)
    assert s["m"]["max"] == 0.21 and s["m"]["within_5pct"] == 0.5
    assert s["z"] == {"geomean": 0.0, "p50": 0.0, "p95": 0.0, "max": 0.0, "within_5pct": 1.0}
