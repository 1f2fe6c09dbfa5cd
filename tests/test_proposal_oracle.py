"""Pins of the FP64 proposal-network oracle: central finite differences of
the loss for every parameter tensor, the max-pool routing rule, and the
Adam update against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import proposal as PR


def _batch(rng, B=3, n=40):
    return [(rng.normal(size=(n, 4)), rng.normal(size=(n, 4))) for _ in range(B)], rng.normal(size=(B, 6))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = PR.init_params(1)
    for k in p:
        if k[0] in "bc":
            p[k] = rng.normal(scale=0.1, size=p[k].shape)
    batch, labels = _batch(rng)
    loss, g = PR.loss_and_grad(p, batch, labels)
    h = 1e-6
    for name, _ in PR.SHAPES:
        idx = [tuple(rng.integers(0, s) for s in p[name].shape) for _ in range(6)]
        for ix in idx:
            old = p[name][ix]
            p[name][ix] = old + h
            lp, _ = PR.loss_and_grad(p, batch, labels)
            p[name][ix] = old - h
            lm, _ = PR.loss_and_grad(p, batch, labels)
            p[name][ix] = old
            fd = (lp - lm) / (2 * h)
            assert g[name][ix] == pytest.approx(fd, rel=1e-4, abs=1e-7), (name, ix)


def test_maxpool_routes_to_argmax():
    rng = np.random.default_rng(1)
    p = PR.init_params(2)
    P = rng.normal(size=(30, 4))
    feat, cache = PR.cloud_feature(p, P)
    h3 = np.maximum(np.maximum(P @ p["W1"].T + p["b1"], 0) @ p["W2"].T + p["b2"], 0) @ p["W3"].T + p["b3"]
    assert np.allclose(feat, h3.max(axis=0))
    assert np.array_equal(cache[-1], h3.argmax(axis=0))


def test_adam_closed_form():
    """On f(x) = x^2 / 2 with g = x, the first Adam step moves every
    coordinate by lr * sign(x) (bias correction makes m_hat / sqrt(v_hat) =
    g / |g|)."""
    p = {"x": np.array([3.0, -0.5, 1e-3])}
    m = {"x": np.zeros(3)}
    v = {"x": np.zeros(3)}
    PR.adam_step(p, {"x": p["x"].copy()}, m, v, 1, lr=0.1, eps=0.0)
    assert np.allclose(p["x"], [2.9, -0.4, 1e-3 - 0.1])
