"""Cost-model network kernels and the autotuner on the GPU.

Gradients of the FP32 kernels are checked against the FP64 CPU oracle
(relative error per parameter tensor <= 1e-4), the Adam kernel against the
oracle's Adam step given the same gradient, and the forward pass against the
oracle's forward pass."""
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
    cj.init(sync=True)
    yield
    cj.shutdown()


def params(F, seed=11, scale=0.5):
    H = 64
    v = synth.uniform_np(seed, 0, H * F + H + H * H + H + H + 1) * scale
    return v.astype(np.float32)


def split(v, F):
    return oracle.MLPParams.from_flat(v.astype(np.float64), F, 64)


@pytest.mark.parametrize("F,B", [(32, 300), (7, 64), (64, 1)])
def test_forward_and_gradient_match_oracle(F, B):
    theta = params(F)
    X = (synth.uniform_np(12, 0, B * F)).astype(np.float32).reshape(B, F)
    t = (synth.uniform_np(13, 0, B) * 2).astype(np.float32)
    net = cj.MLP(F)
    try:
        net.set_params(theta)
        Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
        y = torch.empty(B, device="cuda")
        net.forward(Xd, y)
        g = torch.empty(net.P, device="cuda")
        loss = torch.empty(1, device="cuda")
        net.grad(Xd, td, g, loss)
        torch.cuda.synchronize()
        p64 = split(theta, F)
        y_ref, _, _ = oracle.mlp_forward(p64, X.astype(np.float64))
        np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4)
        loss_ref, g_ref = oracle.mlp_loss_grad(p64, X.astype(np.float64), t.astype(np.float64))
        assert abs(loss.item() - loss_ref) <= 1e-4 * max(1.0, loss_ref)
        got = split(g.cpu().numpy(), F)
        for a, b, name in zip(got.tensors(), g_ref.tensors(), oracle.MLPParams.NAMES):
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
            assert err <= 1e-4, (name, err)
        # parameters unchanged by grad()
        np.testing.assert_array_equal(net.get_params(), theta)
    finally:
        net.destroy()


def test_adam_step_matches_oracle_given_the_same_gradient():
    F, B = 32, 200
    theta = params(F, seed=21)
    X = synth.uniform_np(22, 0, B * F).astype(np.float32).reshape(B, F)
    t = synth.uniform_np(23, 0, B).astype(np.float32)
    net = cj.MLP(F)
    try:
        net.set_params(theta)
        Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
        g = torch.empty(net.P, device="cuda")
        net.grad(Xd, td, g)
        net.train_step(Xd, td, 1e-3)
        torch.cuda.synchronize()
        after = net.get_params().astype(np.float64)
        th = theta.astype(np.float64).copy()
        m = np.zeros_like(th)
        v = np.zeros_like(th)
        oracle.adam(th, g.cpu().numpy().astype(np.float64), m, v, 1, lr=1e-3)
        np.testing.assert_allclose(after, th, rtol=1e-5, atol=1e-6)
    finally:
        net.destroy()


def test_training_reduces_loss_deterministically():
    F, B = 32, 512
    X = synth.uniform_np(31, 0, B * F).astype(np.float32).reshape(B, F)
    t = (X[:, :4].sum(1) + 0.5 * X[:, 5] * X[:, 6]).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    finals = []
    for rep in range(2):
        net = cj.MLP(F, seed=5)
        try:
            loss = torch.empty(1, device="cuda")
            net.grad(Xd, td, torch.empty(net.P, device="cuda"), loss)
            first = loss.item()
            for _ in range(300):
                net.train_step(Xd, td, 3e-3, loss)
            torch.cuda.synchronize()
            finals.append((loss.item(), net.get_params()))
            assert loss.item() < 0.05 * first
        finally:
            net.destroy()
    assert finals[0][0] == finals[1][0]
    np.testing.assert_array_equal(finals[0][1], finals[1][1])


def test_autotune_returns_fastest_candidate_and_all_times():
    n, steps, batch = 8, 16, 4096
    A = synth.chain_inputs_torch(synth.SEED_CHAIN_SWEEP, batch, n, "cuda")
    X = torch.empty_like(A)
    s = torch.cuda.current_stream()
    best, times = cj.autotune(cj.K_UPDATE_CHAIN, cj.F64, cj.chain_launch_vals(A, X, steps), batch, s, reps=3, n=n)
    assert len(times) == len(cj.candidates(cj.K_UPDATE_CHAIN, cj.F64, n=n)) >= 4
    finite = [(tile, ms) for tile, ms in times if np.isfinite(ms)]
    assert len(finite) == len(times)
    assert best == min(finite, key=lambda p: p[1])[0]


def test_cost_model_choice_is_a_candidate():
    net = cj.MLP(cj.FEATURES)
    try:
        net.use_as_cost_model()
        for kw in (dict(kernel=cj.K_UPDATE_CHAIN, dtype=cj.F64, n=24),
                   dict(kernel=cj.K_LTIMES, dtype=cj.F32, layout_a=3, layout_b=1, m=36, d=96)):
            tile, pred = cj.choose_tile(batch=1 << 16, steps=64, **kw)
            k = kw.pop("kernel")
            assert tile in cj.candidates(k, **kw)
            assert np.isfinite(pred)
    finally:
        cj.clear_cost_model()
        net.destroy()
