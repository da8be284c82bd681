"""Pins of the schedule-network oracle: the analytic gradient against central finite
differences of the loss (exact arithmetic, no BF16 rounding), and special cases."""
import numpy as np

from oracle import mlp


def random_params(rng, scale=0.3):
    return rng.normal(scale=scale, size=mlp.NPARAM)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = random_params(rng)
    X = rng.normal(size=(40, 16))
    Y = rng.normal(size=(40, 2))
    L, g = mlp.loss_grad(p, X, Y, bf=False)
    eps = 1e-6
    idx = rng.choice(mlp.NPARAM, size=120, replace=False)
    for k in idx:
        d = np.zeros_like(p)
        d[k] = eps
        fd = (mlp.loss(p + d, X, Y, bf=False) - mlp.loss(p - d, X, Y, bf=False)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd))
    assert L == mlp.loss(p, X, Y, bf=False)


def test_zero_last_layer_outputs_the_bias_and_overshoot_weight():
    rng = np.random.default_rng(1)
    p = random_params(rng)
    P = mlp.unpack(p)
    k = mlp.NPARAM - (2 * 64 + 2)
    p[k:k + 128] = 0.0
    p[-2:] = [1.5, -2.0]
    X = rng.normal(size=(5, 16))
    out = mlp.forward(p, X, bf=False)
    assert np.allclose(out, [[1.5, -2.0]] * 5)
    # overshoot by 1 costs 4, undershoot by 1 costs 1
    assert mlp.loss(p, X, np.tile([0.5, -3.0], (5, 1)), bf=False) == (4.0 + 4.0) / 2
    assert mlp.loss(p, X, np.tile([2.5, -1.0], (5, 1)), bf=False) == (1.0 + 1.0) / 2


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8, -3.0e-5, 65504.0], np.float32)
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                         # tie to even
    assert r[2] == 1.0 + 2 ** -6               # tie to even (upwards)
    assert abs(r[3] - (-3.0e-5)) <= 2 ** -8 * 3.0e-5
    assert r[4] == 65536.0


def test_gradient_tolerance_catches_planted_mistakes():
    """The per-element tolerance the GPU gradient is held to is tight enough to see a
    wrong row, a dropped batch row or a sign error of any block in the oracle's own
    BF16-operand gradient."""
    rng = np.random.default_rng(4)
    p = random_params(rng).astype(np.float32).astype(np.float64)
    X = rng.normal(size=(257, 16)).astype(np.float32).astype(np.float64)
    Y = rng.normal(size=(257, 2)).astype(np.float32).astype(np.float64)
    _, g = mlp.loss_grad(p, X, Y, bf=True)
    tol = mlp.gradient_tolerance(g)
    assert np.all(np.abs(g - g) <= tol)
    blocks = dict(mlp.blocks())
    # two rows of dW1 exchanged
    bad = g.copy()
    w1 = bad[blocks["W1"]].reshape(64, 16)
    w1[[3, 4]] = w1[[4, 3]]
    bad[blocks["W1"]] = w1.ravel()
    assert np.any(np.abs(bad - g) > tol)
    # one batch row left out of the gradient
    _, g_drop = mlp.loss_grad(p, X[1:], Y[1:], bf=True)
    g_drop = g_drop * (X.shape[0] - 1) / X.shape[0]       # same normalisation (mean over 257 rows)
    for name, sl in mlp.blocks():
        assert np.any(np.abs(g_drop[sl] - g[sl]) > tol[sl]), name
    # a sign error in each bias
    for name in ("b1", "b2", "b3"):
        bad = g.copy()
        bad[blocks[name]] *= -1.0
        assert np.any(np.abs(bad - g) > tol), name
