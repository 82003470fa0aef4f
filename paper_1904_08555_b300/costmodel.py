"""Learned cost model: data collection, training and evaluation (harness).

The paper names profiling-guided autotuning of JIT-compiled code as future
work (Sec. 6); this module closes that loop with the library's own pieces:

  1. For each training request, libcj's exhaustive autotuner (cj_autotune)
     compiles every candidate tile and times it on seeded inputs.
  2. Each (request, tile) becomes a feature vector (cj_featurize) with the
     log of its measured time as the target.
  3. The MLP (cj_mlp_*: forward, gradient and Adam kernels on the GPU) is
     trained on that table.
  4. On held-out requests the model's choice (cj_choose_tile: the lowest
     mean predicted log time of an ensemble of networks, the default rule's
     tile kept unless another is predicted 10% faster) is timed against
     exhaustive autotuning: regret = t(chosen) / t(best) - 1.  The same is
     reported for the library's default tile ("no model") and for a uniformly
     random candidate.

Held out means unseen: no held-out request is a training request.  Chain
requests are trained at the sizes TRAIN_CHAIN_N and held out at every other
size in [2, 64]; LTimes requests are trained on 18 of the 36 storage-order
pairs (in, out) and held out on the other 18, split so that every order of in,
every order of out and every combination of their fastest axes appears in
both sets (_lt_split).  BF16 chains (N >= 16) are in both.  evaluate() also runs on the training requests, so the report
separates seen from unseen requests.

Workload sizes: update chain batch = floor(2^22 / N^2), T = 64; LTimes
M = 36, D = 96, G = 32, Z = 2^16.  Everything runs through the C ABI.
"""
from __future__ import annotations

import math
import time

import numpy as np

import synth
from . import cj

T_STEPS = 64
LT_M, LT_D, LT_G, LT_Z = 36, 96, 32, 1 << 16
TRAIN_CHAIN_N = (3, 4, 5, 7, 8, 12, 16, 24, 32, 36, 40, 44, 48, 52, 56, 60, 64)
ENSEMBLE = 16   # networks trained from different seeds; their predictions are averaged


def chain_batch(n: int) -> int:
    return max(1, (1 << 22) // (n * n))


class Request(tuple):
    """(kernel, dtype, n, layout_a, layout_b)."""

    @property
    def kernel(self):
        return self[0]

    def kw(self):
        k, dt, n, la, lb = self
        if k == cj.K_LTIMES:
            return dict(dtype=dt, layout_a=la, layout_b=lb, m=LT_M, d=LT_D)
        return dict(dtype=dt, n=n, layout_a=la)

    def batch(self):
        return LT_G * LT_Z if self[0] == cj.K_LTIMES else chain_batch(self[2])


HELDOUT_CHAIN_N = tuple(n for n in range(2, 65) if n not in TRAIN_CHAIN_N)


def _lt_split():
    """Storage orders by fastest axis: z-fast {0, 2}, g-fast {1, 4}, x-fast
    {3, 5}.  For every (fastest axis of in, fastest axis of out) class of four
    pairs {a, b} x {c, d}, (a, c) and (b, d) are trained and (a, d) and (b, c)
    held out: every class, every order of in and every order of out occurs in
    both sets, while no held-out pair was trained on."""
    fast = ((0, 2), (1, 4), (3, 5))
    train, held = [], []
    for a, b in fast:
        for c, d in fast:
            train += [(a, c), (b, d)]
            held += [(a, d), (b, c)]
    return tuple(sorted(train)), tuple(sorted(held))


TRAIN_LT_PAIRS, HELDOUT_LT_PAIRS = _lt_split()


def training_requests():
    reqs = []
    for dt in (cj.F64, cj.F32, cj.BF16):
        for n in TRAIN_CHAIN_N:
            if dt == cj.BF16 and n < 16:
                continue
            for la in (0, 1):
                reqs.append(Request((cj.K_UPDATE_CHAIN, dt, n, la, 0)))
        if dt != cj.BF16:
            for la, lb in TRAIN_LT_PAIRS:
                reqs.append(Request((cj.K_LTIMES, dt, 0, la, lb)))
    return reqs


def heldout_requests(count: int = 2000, seed: int = synth.SEED_REQUESTS):
    """Seeded stream of unseen requests: kernel chain / LTimes 50/50; chain N
    uniform over the sizes in [2, 64] outside TRAIN_CHAIN_N, layout uniform,
    dtype uniform over those the size supports ({f64, f32}, plus bf16 at
    N >= 16); LTimes order pair uniform over HELDOUT_LT_PAIRS, dtype uniform
    over {f64, f32}."""
    u = [synth.unit_np(seed, synth.STREAM_MISC + j * count, count) for j in range(5)]
    reqs = []
    for i in range(count):
        k = cj.K_UPDATE_CHAIN if u[0][i] < 0.5 else cj.K_LTIMES
        if k == cj.K_UPDATE_CHAIN:
            n = HELDOUT_CHAIN_N[int(u[2][i] * len(HELDOUT_CHAIN_N))]
            dts = (cj.F64, cj.F32, cj.BF16) if n >= 16 else (cj.F64, cj.F32)
            reqs.append(Request((k, dts[int(u[1][i] * len(dts))], n, int(u[3][i] * 2), 0)))
        else:
            dt = cj.F64 if u[1][i] < 0.5 else cj.F32
            la, lb = HELDOUT_LT_PAIRS[int(u[3][i] * len(HELDOUT_LT_PAIRS))]
            reqs.append(Request((k, dt, 0, la, lb)))
    return reqs


class Timer:
    """Exhaustive timings of every candidate of a request (cached)."""

    def __init__(self, reps: int = 3, chain_log2: int = 22):
        import torch
        self.torch = torch
        self.reps = reps
        self.chain_log2 = chain_log2   # chain batch = floor(2^chain_log2 / N^2)
        self.cache = {}
        self.stream = torch.cuda.current_stream()
        self._lt = None

    def _buffers(self, r: Request):
        torch = self.torch
        tdt = torch.float64 if r[1] == cj.F64 else torch.float32   # bf16 chains keep fp32 state
        if r.kernel == cj.K_LTIMES:
            if self._lt is None or self._lt[0] != tdt:
                L, _ = synth.ltimes_inputs_np(synth.SEED_LTIMES, LT_M, LT_D, 1, 1)
                x = synth.uniform_torch(synth.SEED_LTIMES, synth.STREAM_A, LT_D * LT_G * LT_Z, "cuda").to(tdt)
                out = torch.empty(LT_M * LT_G * LT_Z, device="cuda", dtype=tdt)
                self._lt = (tdt, torch.from_numpy(L).to("cuda", tdt), x, out)
            _, L, x, out = self._lt
            # the storage order only changes addressing; the same buffer serves every order
            return cj.ltimes_launch_vals(L, x, out, LT_G, LT_Z), (L, x, out)
        n = r[2]
        b = self.batch(r)
        A = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").to(tdt)
        X = torch.empty_like(A)
        return cj.chain_launch_vals(A, X, T_STEPS), (A, X)

    def batch(self, r: Request) -> int:
        return r.batch() if r.kernel == cj.K_LTIMES else max(1, (1 << self.chain_log2) // (r[2] * r[2]))

    def prefetch(self, reqs):
        """Queue every candidate's compile (async mode: parallel background threads)."""
        for r in set(reqs):
            for tile in cj.candidates(r.kernel, **r.kw()):
                cj.specialize(r.kernel, tile=tile, flags=cj.FLAG_NO_AOT, **r.kw())

    def times(self, r: Request):
        if r in self.cache:
            return self.cache[r]
        vals, keep = self._buffers(r)
        _, tt = cj.autotune(r.kernel, launch_vals=vals, batch=self.batch(r), stream=self.stream, reps=self.reps,
                            **r.kw())
        del keep
        self.cache[r] = dict(tt)
        return self.cache[r]

    def time_tile(self, r: Request, tile):
        """Time one tile (e.g. the default) the same way the autotuner does."""
        t = self.times(r)
        if tuple(tile) in t:
            return t[tuple(tile)]
        torch = self.torch
        _, keep = self._buffers(r)
        h = cj.specialize(r.kernel, tile=tile, **r.kw())
        h.wait(-1)
        ms = []
        launch = (lambda: cj.launch_update_chain(h, keep[0], keep[1], T_STEPS, batch=self.batch(r), stream=self.stream)) \
            if r.kernel != cj.K_LTIMES else \
            (lambda: cj.launch_ltimes(h, keep[0], keep[1], keep[2], LT_G, LT_Z, stream=self.stream))
        launch()
        for _ in range(self.reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            launch()
            e1.record(self.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        del keep
        t[tuple(tile)] = float(np.median(ms))
        return t[tuple(tile)]


def default_tile(r: Request):
    """The library's default tile for this request (from its canonical key)."""
    h = cj.specialize(r.kernel, **r.kw())
    key = bytes.fromhex(h.key_hex)
    return tuple(int.from_bytes(key[12 + 4 * i:16 + 4 * i], "little") for i in range(4))


def dataset(timer: Timer, reqs):
    X, y, meta = [], [], []
    for r in reqs:
        for tile, ms in timer.times(r).items():
            if not math.isfinite(ms) or ms <= 0:
                continue
            X.append(cj.featurize(r.kernel, batch=r.batch(), steps=T_STEPS, tile=tile, **r.kw()))
            y.append(math.log(ms))
            meta.append((r, tile))
    return np.array(X, dtype=np.float32), np.array(y, dtype=np.float64), meta


class CostModel:
    """An ensemble of ENSEMBLE networks, each trained on the same table from
    its own initial weights; the library averages their predictions.  Each
    network predicts the natural log of the time in ms."""

    def __init__(self, seed: int = synth.SEED_REQUESTS, members: int = ENSEMBLE):
        self.nets = [cj.MLP(cj.FEATURES, seed=seed + 7919 * i) for i in range(members)]
        self.losses = []

    def fit(self, X, y, steps: int = 4000, lr: float = 2e-3):
        """Adam with cosine decay on the standardised log time, then the
        standardisation folded into each network's output layer."""
        torch = __import__("torch")
        mu, sd = float(y.mean()), float(y.std() + 1e-9)
        Xd = torch.from_numpy(X).cuda()
        td = torch.from_numpy(((y - mu) / sd).astype(np.float32)).cuda()
        loss = torch.empty(1, device="cuda")
        F = X.shape[1]
        w3 = F * 64 + 64 + 64 * 64 + 64
        finals = []
        for net in self.nets:
            for s in range(steps):
                cur = lr * 0.5 * (1 + math.cos(math.pi * s / steps)) + 1e-5
                net.train_step(Xd, td, cur, loss)
                if s % 1000 == 0 or s == steps - 1:
                    torch.cuda.synchronize()
                    self.losses.append((len(finals), s, loss.item()))
            torch.cuda.synchronize()
            finals.append(self.losses[-1][2])
            p = net.get_params()
            p[w3:w3 + 64] *= sd
            p[w3 + 64] = p[w3 + 64] * sd + mu
            net.set_params(p)
        return float(np.mean(finals))

    def predict(self, X):
        torch = __import__("torch")
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        y = torch.empty(X.shape[0], device="cuda")
        out = np.zeros(X.shape[0])
        for net in self.nets:
            net.forward(Xd, y)
            out += y.cpu().numpy()
        return out / len(self.nets)

    def install(self):
        cj.use_cost_model_ensemble(self.nets)

    def destroy(self):
        cj.clear_cost_model()
        for net in self.nets:
            net.destroy()


def evaluate(model: CostModel, timer: Timer, reqs, seed: int = 7):
    """Regret of the model's choice, the default tile and a random candidate."""
    model.install()
    rng = np.random.default_rng(seed)
    out = {"model": [], "default": [], "random": []}
    picks = {}
    for r in reqs:
        t = timer.times(r)
        best = min(v for v in t.values() if math.isfinite(v))
        if r not in picks:
            tile, _ = cj.choose_tile(r.kernel, batch=r.batch(), steps=T_STEPS, **r.kw())
            picks[r] = (tile, default_tile(r))
        tile, dflt = picks[r]
        out["model"].append(timer.time_tile(r, tile) / best - 1.0)
        out["default"].append(timer.time_tile(r, dflt) / best - 1.0)
        finite = [v for v in t.values() if math.isfinite(v)]
        out["random"].append(finite[rng.integers(len(finite))] / best - 1.0)
    return {k: np.array(v) for k, v in out.items()}


def summarize(reg):
    def gm(v):
        return float(np.exp(np.mean(np.log1p(v))) - 1.0)
    return {k: {"geomean": gm(v), "p50": float(np.percentile(v, 50)), "p95": float(np.percentile(v, 95)),
                "max": float(v.max()), "within_5pct": float(np.mean(v <= 0.05))} for k, v in reg.items()}


def ranking_check(small: Timer, reqs, chain_log2: int = 25):
    """Do the reduced timing sizes rank the candidates as the configs' own
    sizes do?  For chain requests, every candidate is timed again at batch
    floor(2^chain_log2 / N^2): Spearman's rank correlation of the two
    timings, whether the fastest candidate agrees, and the regret at the
    large size of the candidate that is fastest at the small one."""
    big = Timer(reps=small.reps, chain_log2=chain_log2)
    rows = []
    for r in reqs:
        a, b = small.times(r), big.times(r)
        tiles = [t for t in a if math.isfinite(a[t]) and math.isfinite(b.get(t, math.inf))]
        ra = np.argsort(np.argsort([a[t] for t in tiles]))
        rb = np.argsort(np.argsort([b[t] for t in tiles]))
        rho = float(np.corrcoef(ra, rb)[0, 1]) if len(tiles) > 2 else 1.0
        best_small = min(tiles, key=lambda t: a[t])
        best_big = min(tiles, key=lambda t: b[t])
        rows.append({"request": list(r), "candidates": len(tiles), "spearman": rho,
                     "same_fastest": best_small == best_big,
                     "regret_at_large_of_small_fastest": b[best_small] / b[best_big] - 1.0})
    return {"chain_batch_small": f"2^{small.chain_log2}/N^2", "chain_batch_large": f"2^{chain_log2}/N^2",
            "requests": rows,
            "mean_spearman": float(np.mean([x["spearman"] for x in rows])),
            "same_fastest_share": float(np.mean([x["same_fastest"] for x in rows])),
            "max_regret_at_large": float(max(x["regret_at_large_of_small_fastest"] for x in rows))}


def run(n_heldout: int = 2000, train_steps: int = 4000, reps: int = 3, log=print):
    """Full procedure; returns a result dict (used by bench.py --workload costmodel)."""
    t0 = time.perf_counter()
    timer = Timer(reps=reps)
    train = training_requests()
    held = heldout_requests(n_heldout)
    timer.prefetch(train + held)
    X, y, _ = dataset(timer, train)
    t_collect = time.perf_counter() - t0
    log(f"training table: {len(y)} rows from {len(train)} requests ({t_collect:.1f} s)")
    model = CostModel()
    t1 = time.perf_counter()
    final = model.fit(X, y, steps=train_steps)
    t_train = time.perf_counter() - t1
    pred = model.predict(X)
    fit_rmse = float(np.sqrt(np.mean((pred - y) ** 2)))
    log(f"trained {train_steps} Adam steps on the GPU in {t_train:.1f} s, loss {final:.4f}, rmse(log ms) {fit_rmse:.3f}")
    assert not set(held) & set(train), "held-out requests must be unseen"
    reg = evaluate(model, timer, held)
    summ = summarize(reg)
    by_kind = {}
    for name, pick in (("chain", lambda r: r.kernel == cj.K_UPDATE_CHAIN and r[1] != cj.BF16),
                       ("chain_bf16", lambda r: r[1] == cj.BF16), ("ltimes", lambda r: r.kernel == cj.K_LTIMES)):
        mask = np.array([pick(r) for r in held])
        if mask.any():
            by_kind[name] = summarize({k: v[mask] for k, v in reg.items()})
    seen = summarize(evaluate(model, timer, train))
    # a subset of chain requests re-timed at the configs' own batch 2^25/N^2
    subset = [Request((cj.K_UPDATE_CHAIN, dt, n, 0, 0)) for dt in (cj.F64, cj.F32) for n in (5, 13, 27, 50)]
    subset += [Request((cj.K_UPDATE_CHAIN, cj.BF16, n, 0, 0)) for n in (27, 50)]
    t2 = time.perf_counter()
    ranking = ranking_check(timer, subset)
    log(f"ranking check at 2^25/N^2 on {len(subset)} requests: {time.perf_counter() - t2:.1f} s")
    distinct = len(set(held))
    ncand = [len(cj.candidates(r.kernel, **r.kw())) for r in set(held)]
    model.destroy()
    return {"heldout_requests": len(held), "distinct_heldout": distinct, "train_rows": int(len(y)),
            "train_requests": len(train), "fit_rmse_log_ms": fit_rmse, "train_seconds": t_train,
            "collect_seconds": t_collect, "regret": summ, "regret_unseen_by_kind": by_kind,
            "regret_seen_training_requests": seen, "ranking_check": ranking,
            "compiles_per_request": {"model": 1, "exhaustive_mean": float(np.mean(ncand))},
            "losses": model.losses}
