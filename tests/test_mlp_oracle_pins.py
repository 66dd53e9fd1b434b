"""Pins of the FP64 surrogate-MLP oracle (no GPU)."""
import numpy as np

from oracle import mlp


def _rand_params(rng, d_in, h1, h2, scale=0.5):
    s = mlp.sizes(d_in, h1, h2)
    return mlp.flatten({k: rng.normal(0, scale, shp) for k, shp in s.items()})


def test_finite_differences():
    rng = np.random.default_rng(0)
    d_in, h1, h2 = 7, 9, 5
    p = _rand_params(rng, d_in, h1, h2)
    x = rng.normal(size=(13, d_in))
    t = rng.normal(size=13)
    _, g = mlp.grad(p, x, t, d_in, h1, h2)
    h = 1e-6
    for i in rng.choice(len(p), 40, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, t, d_in=d_in, h1=h1, h2=h2) - mlp.loss(p - e, x, t, d_in=d_in, h1=h1, h2=h2)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_one_hidden_unit_closed_form():
    # y = w3 * relu(w2 * relu(w1 . x + b1) + b2) + b3 with all pre-activations positive
    w1 = np.array([[0.5, -0.25, 1.0]])
    b1 = np.array([0.1])
    w2 = np.array([[2.0]])
    b2 = np.array([0.3])
    w3 = np.array([1.5])
    b3 = np.array([-0.2])
    p = mlp.flatten({"W1": w1, "b1": b1, "W2": w2, "b2": b2, "w3": w3, "b3": b3})
    x = np.array([[1.0, 0.0, 2.0]])
    a1 = 0.5 + 2.0 + 0.1            # 2.6
    a2 = 2.0 * a1 + 0.3             # 5.5
    y_expect = 1.5 * a2 - 0.2       # 8.05
    y, _ = mlp.forward(p, x, 3, 1, 1)
    assert abs(y[0] - y_expect) < 1e-12
    t = np.array([1.0])
    l, g = mlp.grad(p, x, t, 3, 1, 1)
    dy = 2 * (y_expect - 1.0)
    G = mlp.unflatten(g, 3, 1, 1)
    assert abs(l - (y_expect - 1.0) ** 2) < 1e-12
    assert abs(G["b3"][0] - dy) < 1e-12
    assert abs(G["w3"][0] - dy * a2) < 1e-12
    assert abs(G["b2"][0] - dy * 1.5) < 1e-12
    assert abs(G["W2"][0, 0] - dy * 1.5 * a1) < 1e-12
    assert abs(G["b1"][0] - dy * 1.5 * 2.0) < 1e-12
    assert np.allclose(G["W1"][0], dy * 1.5 * 2.0 * x[0], atol=1e-12)


def test_relu_cuts_the_gradient():
    # a hidden unit that is off everywhere gets no gradient
    rng = np.random.default_rng(3)
    p = _rand_params(rng, 4, 3, 2)
    P = mlp.unflatten(p, 4, 3, 2)
    P["W1"][1] = 0.0
    P["b1"][1] = -1.0
    p = mlp.flatten(P)
    x = rng.normal(size=(8, 4))
    _, g = mlp.grad(p, x, rng.normal(size=8), 4, 3, 2)
    G = mlp.unflatten(g, 4, 3, 2)
    assert np.all(G["W1"][1] == 0) and G["b1"][1] == 0 and np.all(G["W2"][:, 1] == 0)


def test_linear_regime_matches_least_squares_gradient():
    # with every pre-activation positive the net is affine: y = A x + c
    rng = np.random.default_rng(4)
    d_in, h1, h2 = 5, 6, 4
    P = {"W1": np.abs(rng.normal(size=(h1, d_in))), "b1": np.full(h1, 5.0),
         "W2": np.abs(rng.normal(size=(h2, h1))), "b2": np.full(h2, 5.0),
         "w3": rng.normal(size=h2), "b3": np.array([0.3])}
    p = mlp.flatten(P)
    x = np.abs(rng.normal(size=(10, d_in)))
    y, _ = mlp.forward(p, x, d_in, h1, h2)
    A = P["w3"] @ P["W2"] @ P["W1"]
    c = P["w3"] @ (P["W2"] @ P["b1"] + P["b2"]) + P["b3"][0]
    assert np.allclose(y, x @ A + c, rtol=1e-12)


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.0 + 2 ** -8 + 2 ** -9, -3.14159, 0.0], dtype=np.float32)
    r = mlp.round_bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0            # tie (halfway) rounds to even
    assert r[2] == 1.0078125      # above halfway rounds up
    assert abs(r[3] + 3.140625) < 1e-12
    assert r[4] == 0.0
