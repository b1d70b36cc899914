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
