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
    # 50/50 kernels: binomial(2000, 1/2) has sd 22.4; 5 sd either side
    assert abs(len(chains) - 1000) < 112
    assert abs(sum(r[1] == cj.F64 for r in lt) - len(lt) / 2) < 5 * (len(lt) / 4) ** 0.5
    assert {r[1] for r in chains} == {cj.F64, cj.F32, cj.BF16} and {r[1] for r in lt} == {cj.F64, cj.F32}
    assert all(r[2] >= 16 for r in chains if r[1] == cj.BF16)
    assert {r[2] for r in chains} == set(costmodel.HELDOUT_CHAIN_N)
    assert min(r[2] for r in chains) == 2 and max(r[2] for r in chains) == 63
    assert {r[3] for r in chains} == {0, 1} and all(r[4] == 0 for r in chains)
    assert {(r[3], r[4]) for r in lt} == set(costmodel.HELDOUT_LT_PAIRS)
    assert all(r[2] == 0 for r in lt)


def test_heldout_requests_are_unseen():
    """No held-out request is a training request: the chain sizes and the
    LTimes order pairs of the two sets are disjoint, while every storage
    order of `in` and of `out` occurs in both."""
    train = set(costmodel.training_requests())
    held = set(costmodel.heldout_requests(2000))
    assert not train & held
    assert not set(costmodel.TRAIN_CHAIN_N) & set(costmodel.HELDOUT_CHAIN_N)
    assert set(costmodel.TRAIN_CHAIN_N) | set(costmodel.HELDOUT_CHAIN_N) == set(range(2, 65))
    assert not set(costmodel.TRAIN_LT_PAIRS) & set(costmodel.HELDOUT_LT_PAIRS)
    fastest = {0: "z", 2: "z", 1: "g", 4: "g", 3: "x", 5: "x"}    # fastest axis of each storage order
    for pairs in (costmodel.TRAIN_LT_PAIRS, costmodel.HELDOUT_LT_PAIRS):
        assert len(pairs) == 18
        assert {i for i, _ in pairs} == set(range(6)) and {o for _, o in pairs} == set(range(6))
        assert {(fastest[i], fastest[o]) for i, o in pairs} == {(a, b) for a in "zgx" for b in "zgx"}


def test_training_requests_cover_every_dtype_size_and_order():
    t = costmodel.training_requests()
    n_bf16 = sum(n >= 16 for n in costmodel.TRAIN_CHAIN_N)
    assert len(t) == 2 * (len(costmodel.TRAIN_CHAIN_N) * 2 + 18) + 2 * n_bf16
    assert len(set(t)) == len(t)
    for dt in (cj.F64, cj.F32):
        assert {(r[3], r[4]) for r in t if r.kernel == cj.K_LTIMES and r[1] == dt} == set(costmodel.TRAIN_LT_PAIRS)
        assert {r[2] for r in t if r.kernel == cj.K_UPDATE_CHAIN and r[1] == dt} == set(costmodel.TRAIN_CHAIN_N)
    assert {r[2] for r in t if r[1] == cj.BF16} == {n for n in costmodel.TRAIN_CHAIN_N if n >= 16}


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
