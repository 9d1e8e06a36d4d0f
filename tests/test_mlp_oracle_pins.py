"""Pins of the MLP oracle: its backpropagation against central finite
differences, its BF16 rounding against hand values, its Adam step against the
update formula written out for one scalar."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_hand_values():
    x = np.array([1.0, 1.00390625, 1.0 + 2 ** -8 + 2 ** -9, 3.14159265, -2.0 ** -130], np.float32)
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                     # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa
    assert r[2] == 1.0 + 2 ** -7           # above the tie: rounds up
    assert r[3] == 3.140625
    assert r[4] == np.float32(-2.0 ** -130)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    feat = rng.standard_normal((16, mlp.F)) * 2 + 1
    target = rng.uniform(0, 16, 16)
    p = mlp.init_params(3, feat.mean(0), feat.std(0) + 0.1).astype(np.float64)
    p[mlp.OFF_B1:mlp.OFF_W2] = 0.1
    p[mlp.OFF_B2:mlp.OFF_W3] = 0.1
    loss, g = mlp.grad(p, feat, target, round_bf16=False)
    idx = np.concatenate([rng.choice(np.arange(mlp.OFF_W1, mlp.NPARAM), 60, replace=False), [mlp.OFF_B3]])
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        lp = np.mean((mlp.forward(pp, feat, False)[0] - target) ** 2)
        lm = np.mean((mlp.forward(pm, feat, False)[0] - target) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])
    assert np.all(g[:mlp.OFF_W1] == 0)


def test_adam_step_formula():
    p = np.zeros(mlp.NPARAM)
    m = np.zeros(mlp.NPARAM)
    v = np.zeros(mlp.NPARAM)
    g = np.zeros(mlp.NPARAM)
    g[mlp.OFF_B3] = 0.5
    p2, m2, v2 = mlp.adam_step(p, m, v, g, 1, 1e-2)
    # first step: mhat = g, vhat = g^2 -> update = lr * g / (|g| + eps)
    assert abs(p2[mlp.OFF_B3] - (-1e-2 * 0.5 / (0.5 + 1e-8))) < 1e-15
    assert np.count_nonzero(p2) == 1
