"""Plain FP64 numpy oracle of the block-rank MLP (TEST INFRASTRUCTURE ONLY).

32 standardised features -> 64 -> 64 -> 1 with ReLU, weights rounded to BF16
(round to nearest even) in the forward and backward passes, mean squared error,
gradients with respect to the FP32 master weights (straight-through), Adam
(beta1 0.9, beta2 0.999, eps 1e-8).  Written from the textbook definitions of
backpropagation and Adam (Kingma & Ba, 2015); it shares no code with the CUDA
training kernels.
Parameter layout: [mu 32][sigma 32][W1 64x32][b1 64][W2 64x64][b2 64][W3 64][b3 1].
"""
import numpy as np

F, H = 32, 64
OFF_MU, OFF_SIG, OFF_W1 = 0, F, 2 * F
OFF_B1 = OFF_W1 + H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAM = OFF_B3 + 1


def bf16(x):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, round_bf16=True):
    """Weights as used by the network: BF16-rounded float32 masters, or the
    values themselves (float64) when round_bf16 is off."""
    w = bf16(np.asarray(p, np.float32)) if round_bf16 else np.asarray(p, np.float64)
    return dict(mu=w[OFF_MU:OFF_SIG] if not round_bf16 else np.asarray(p, np.float32)[OFF_MU:OFF_SIG].astype(np.float64),
                sig=w[OFF_SIG:OFF_W1] if not round_bf16 else np.asarray(p, np.float32)[OFF_SIG:OFF_W1].astype(np.float64),
                W1=w[OFF_W1:OFF_B1].reshape(H, F), b1=w[OFF_B1:OFF_W2],
                W2=w[OFF_W2:OFF_B2].reshape(H, H), b2=w[OFF_B2:OFF_W3],
                W3=w[OFF_W3:OFF_B3], b3=w[OFF_B3])


def forward(p, feat, round_bf16=True):
    m = unpack(p, round_bf16)
    z = (np.asarray(feat, np.float64) - m["mu"]) / m["sig"]
    a1 = z @ m["W1"].T + m["b1"]
    h1 = np.maximum(a1, 0)
    a2 = h1 @ m["W2"].T + m["b2"]
    h2 = np.maximum(a2, 0)
    y = h2 @ m["W3"] + m["b3"]
    return y, (z, a1, h1, a2, h2)


def grad(p, feat, target, round_bf16=True):
    """Loss (mean squared error) and its gradient with respect to every parameter."""
    m = unpack(p, round_bf16)
    y, (z, a1, h1, a2, h2) = forward(p, feat, round_bf16)
    t = np.asarray(target, np.float64)
    B = y.shape[0]
    loss = np.mean((y - t) ** 2)
    dy = 2 * (y - t) / B
    g = np.zeros(NPARAM)
    g[OFF_W3:OFF_B3] = h2.T @ dy
    g[OFF_B3] = dy.sum()
    d2 = np.outer(dy, m["W3"]) * (a2 > 0)
    g[OFF_W2:OFF_B2] = (d2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(0)
    d1 = (d2 @ m["W2"]) * (a1 > 0)
    g[OFF_W1:OFF_B1] = (d1.T @ z).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(0)
    return loss, g


def adam_step(p, m, v, g, t, lr):
    """One Adam step at step number t (1-based); mu and sigma are not trained."""
    p = np.asarray(p, np.float64).copy()
    m = 0.9 * m + 0.1 * g
    v = 0.999 * v + 0.001 * g * g
    upd = lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    upd[:OFF_W1] = 0
    return p - upd, m, v


def init_params(seed, mu, sigma):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.Generator(np.random.Philox(seed))
    p = np.zeros(NPARAM, np.float32)
    p[OFF_MU:OFF_SIG] = mu
    p[OFF_SIG:OFF_W1] = sigma
    p[OFF_W1:OFF_B1] = rng.standard_normal(H * F) * np.sqrt(2.0 / F)
    p[OFF_W2:OFF_B2] = rng.standard_normal(H * H) * np.sqrt(2.0 / H)
    p[OFF_W3:OFF_B3] = rng.standard_normal(H) * np.sqrt(1.0 / H)
    return p
