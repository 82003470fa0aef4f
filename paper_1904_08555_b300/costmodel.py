"""Learned cost model: data collection, training and evaluation (harness).

The paper names profiling-guided autotuning of JIT-compiled code as future
work (Sec. 6); this module closes that loop with the library's own pieces:

  1. For each training request, libcj's exhaustive autotuner (cj_autotune)
     compiles every candidate tile and times it on seeded inputs.
  2. Each (request, tile) becomes a feature vector (cj_featurize) with the
     log of its measured time as the target.
  3. The MLP (cj_mlp_*: forward, gradient and Adam kernels on the GPU) is
     trained on that table.
  4. On held-out requests the model's choice (cj_choose_tile, argmin of the
     predicted log time over the candidates) is timed against exhaustive
     autotuning: regret = t(chosen) / t(best) - 1.  The same is reported for
     the library's default tile ("no model") and for a uniformly random
     candidate.

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
TRAIN_CHAIN_N = (3, 4, 5, 7, 8, 12, 16, 24, 32, 40, 48, 56, 64)


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


def training_requests():
    reqs = []
    for dt in (cj.F64, cj.F32):
        for n in TRAIN_CHAIN_N:
            for la in (0, 1):
                reqs.append(Request((cj.K_UPDATE_CHAIN, dt, n, la, 0)))
        for la in range(6):
            for lb in range(6):
                reqs.append(Request((cj.K_LTIMES, dt, 0, la, lb)))
    return reqs


def heldout_requests(count: int = 2000, seed: int = synth.SEED_REQUESTS):
    """Seeded stream: kernel chain / LTimes 50/50, N uniform in [2, 64],
    storage orders uniform, dtype uniform over {f64, f32}."""
    u = [synth.unit_np(seed, synth.STREAM_MISC + j * count, count) for j in range(5)]
    reqs = []
    for i in range(count):
        k = cj.K_UPDATE_CHAIN if u[0][i] < 0.5 else cj.K_LTIMES
        dt = cj.F64 if u[1][i] < 0.5 else cj.F32
        if k == cj.K_UPDATE_CHAIN:
            n = 2 + int(u[2][i] * 63)
            reqs.append(Request((k, dt, n, int(u[3][i] * 2), 0)))
        else:
            reqs.append(Request((k, dt, 0, int(u[3][i] * 6), int(u[4][i] * 6))))
    return reqs


class Timer:
    """Exhaustive timings of every candidate of a request (cached)."""

    def __init__(self, reps: int = 3):
        import torch
        self.torch = torch
        self.reps = reps
        self.cache = {}
        self.stream = torch.cuda.current_stream()
        self._lt = None

    def _buffers(self, r: Request):
        torch = self.torch
        tdt = torch.float64 if r[1] == cj.F64 else torch.float32
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
        b = chain_batch(n)
        A = synth.uniform_torch(synth.SEED_CHAIN_SWEEP, synth.STREAM_A, b * n * n, "cuda").to(tdt)
        X = torch.empty_like(A)
        return cj.chain_launch_vals(A, X, T_STEPS), (A, X)

    def prefetch(self, reqs):
        """Queue every candidate's compile (async mode: parallel background threads)."""
        for r in set(reqs):
            for tile in cj.candidates(r.kernel, **r.kw()):
                cj.specialize(r.kernel, tile=tile, flags=cj.FLAG_NO_AOT, **r.kw())

    def times(self, r: Request):
        if r in self.cache:
            return self.cache[r]
        vals, keep = self._buffers(r)
        _, tt = cj.autotune(r.kernel, launch_vals=vals, batch=r.batch(), stream=self.stream, reps=self.reps,
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
        launch = (lambda: cj.launch_update_chain(h, keep[0], keep[1], T_STEPS, batch=r.batch(), stream=self.stream)) \
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
    """Trained network plus the target standardisation used in training."""

    def __init__(self, seed: int = synth.SEED_REQUESTS):
        self.net = cj.MLP(cj.FEATURES, seed=seed)
        self.mu, self.sd = 0.0, 1.0
        self.losses = []

    def fit(self, X, y, steps: int = 4000, lr: float = 2e-3):
        torch = __import__("torch")
        self.mu, self.sd = float(y.mean()), float(y.std() + 1e-9)
        Xd = torch.from_numpy(X).cuda()
        td = torch.from_numpy(((y - self.mu) / self.sd).astype(np.float32)).cuda()
        loss = torch.empty(1, device="cuda")
        for s in range(steps):
            # cosine learning-rate decay
            cur = lr * 0.5 * (1 + math.cos(math.pi * s / steps)) + 1e-5
            self.net.train_step(Xd, td, cur, loss)
            if s % 500 == 0 or s == steps - 1:
                torch.cuda.synchronize()
                self.losses.append((s, loss.item()))
        torch.cuda.synchronize()
        return self.losses[-1][1]

    def predict(self, X):
        torch = __import__("torch")
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        y = torch.empty(X.shape[0], device="cuda")
        self.net.forward(Xd, y)
        return y.cpu().numpy() * self.sd + self.mu

    def install(self):
        self.net.use_as_cost_model()

    def destroy(self):
        cj.clear_cost_model()
        self.net.destroy()


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
    reg = evaluate(model, timer, held)
    summ = summarize(reg)
    distinct = len(set(held))
    ncand = [len(cj.candidates(r.kernel, **r.kw())) for r in set(held)]
    model.destroy()
    return {"heldout_requests": len(held), "distinct_heldout": distinct, "train_rows": int(len(y)),
            "train_requests": len(train), "fit_rmse_log_ms": fit_rmse, "train_seconds": t_train,
            "collect_seconds": t_collect, "regret": summ,
            "compiles_per_request": {"model": 1, "exhaustive_mean": float(np.mean(ncand))},
            "losses": model.losses}
