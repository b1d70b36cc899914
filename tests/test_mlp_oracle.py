"""Pin of the fp64 cost-network oracle: its hand-written gradient equals
central finite differences of its loss."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, size=mlp.NPARAMS)
    x = rng.normal(size=(20, mlp.F))
    y = rng.normal(size=20)
    loss, g = mlp.loss_and_grad(p, x, y)
    eps = 1e-6
    idx = rng.choice(mlp.NPARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAMS - 1, 0, 12 * 64 + 3]])
    for k in idx:
        e = np.zeros_like(p)
        e[k] = eps
        fd = (mlp.loss_and_grad(p + e, x, y)[0] - mlp.loss_and_grad(p - e, x, y)[0]) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(fd)), k


def test_forward_closed_form_linear_regime():
    # with all pre-activations positive the network is affine in x
    rng = np.random.default_rng(1)
    p = np.abs(rng.normal(0, 0.1, size=mlp.NPARAMS))
    x = np.abs(rng.normal(size=(5, mlp.F)))
    w = mlp.unpack(p)
    want = ((x @ w["W1"].T + w["b1"]) @ w["W2"].T + w["b2"]) @ w["w3"] + w["b3"][0]
    got, _ = mlp.forward(p, x)
    assert np.allclose(got, want, rtol=1e-12)


def test_adam_first_step_has_size_lr():
    """Kingma and Ba: with zero moments, the bias-corrected first step is
    lr * g / (|g| + eps) -- a step of about lr against the gradient's sign."""
    g = np.array([2.0, -0.5, 1e-3, 0.0])
    p, m1, m2 = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-18)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)


def test_adam_scalar_steps_by_hand():
    """f(x) = x^2 from x = 1 with lr = 0.1, two steps worked by hand:
    step 1: g = 2, m1 = 0.2, m2 = 0.004, mhat = 2, vhat = 4, x = 1 - 0.1 * 2 / (2 + eps);
    step 2: g = 2 x1, m1 = 0.9 * 0.2 + 0.1 g, m2 = 0.999 * 0.004 + 0.001 g^2,
            mhat = m1 / 0.19, vhat = m2 / 0.001999."""
    eps = 1e-8
    x1 = 1.0 - 0.1 * 2.0 / (2.0 + eps)
    g2 = 2.0 * x1
    m1 = 0.9 * 0.2 + 0.1 * g2
    m2 = 0.999 * 0.004 + 0.001 * g2 * g2
    x2 = x1 - 0.1 * (m1 / 0.19) / (np.sqrt(m2 / 0.001999) + eps)
    p, a, b = np.array([1.0]), np.zeros(1), np.zeros(1)
    for t in (1, 2):
        p, a, b = mlp.adam_step(p, 2.0 * p, a, b, t, 0.1)
        if t == 1:
            assert abs(p[0] - x1) < 1e-15
    assert abs(p[0] - x2) < 1e-15


def test_adam_training_reduces_loss_and_records_gradients():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(64, mlp.F))
    y = x[:, 0] - 2.0 * x[:, 5]
    p0 = rng.normal(0, 0.2, size=mlp.NPARAMS)
    l0, g0 = mlp.loss_and_grad(p0, x, y)
    p, loss, grads = mlp.train(p0, x, y, steps=200, lr=3e-3)
    assert grads.shape == (200, mlp.NPARAMS) and np.array_equal(grads[0], g0)
    assert loss < 0.2 * l0
