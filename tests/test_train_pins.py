"""Pins of the training-step oracle (activations, their chain rule, Adam) against closed forms,
finite differences and PyTorch's own Adam."""
import numpy as np
import pytest

from oracle import train as T


def test_activations_at_known_points():
    s, o = T.activate([0.0, np.log(2.5)], [0.0, np.log(3.0)])
    np.testing.assert_allclose(s, [1.0, 2.5], rtol=1e-15)
    np.testing.assert_allclose(o, [0.5, 0.75], rtol=1e-15)


def test_chain_rule_matches_central_differences():
    rng = np.random.default_rng(0)
    x = rng.normal(-3.0, 1.0, 50)
    y = rng.normal(0.0, 2.0, 50)
    ws = rng.normal(size=50)
    wo = rng.normal(size=50)

    def loss(x_, y_):
        s, o = T.activate(x_, y_)
        return float((ws * s).sum() + (wo * o).sum())

    gx, gy = T.chain(x, y, ws, wo)
    h = 1e-6
    for i in range(0, 50, 7):
        e = np.zeros(50)
        e[i] = h
        assert gx[i] == pytest.approx((loss(x + e, y) - loss(x - e, y)) / (2 * h), rel=1e-6, abs=1e-12)
        assert gy[i] == pytest.approx((loss(x, y + e) - loss(x, y - e)) / (2 * h), rel=1e-6, abs=1e-12)


def test_adam_first_step_is_a_signed_learning_rate():
    # t = 1 from zero moments: m_hat = g, v_hat = g^2, so the step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m, v = T.adam(np.ones(4), g, np.zeros(4), np.zeros(4), 1, 0.01, eps=1e-15)
    np.testing.assert_allclose(p, 1.0 - 0.01 * g / (np.abs(g) + 1e-15), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)  # 1 - b1 and 1 - b2 round in FP64
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


@pytest.mark.parametrize("eps", [1e-15, 1e-8])
def test_adam_matches_torch_adam_over_several_steps(eps):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p0 = [rng.normal(size=40), rng.normal(size=(10, 3))]
    lrs = [1.6e-4, 5e-3]
    tp = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in p0]
    opt = torch.optim.Adam([{"params": [t], "lr": lr} for t, lr in zip(tp, lrs)], betas=(0.9, 0.999), eps=eps)
    ours = [(a.copy(), np.zeros_like(a), np.zeros_like(a)) for a in p0]
    for step in range(1, 6):
        grads = [rng.normal(size=a.shape) * (1 + step) for a in p0]
        for t, g in zip(tp, grads):
            t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        ours = [T.adam(p, g, m, v, step, lr, eps=eps) for (p, m, v), g, lr in zip(ours, grads, lrs)]
        for (p, _, _), t in zip(ours, tp):
            np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-15)
