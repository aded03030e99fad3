"""Pins of the FP64 reference network: the analytic gradient against central finite
differences (pure FP64), BF16 rounding against exactly representable values, and the
forward pass against a plain per-sample loop."""
import numpy as np

from oracle import mlp


def _setup(seed=0, n=40):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.N_PARAMS)
    norm = np.concatenate([rng.normal(0, 1, 6), rng.uniform(0.5, 2, 6), [1.2, 0.4]])
    X = rng.normal(0, 1, (n, 6)) * norm[6:12] + norm[0:6]
    logT = rng.normal(1.2, 0.4, n)
    return p, norm, X, logT


def test_gradient_matches_finite_differences():
    p, norm, X, logT = _setup()
    _, g = mlp.loss_and_grad(p, norm, X, logT, bf16=False)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(np.arange(0, 384), 8), rng.choice(np.arange(384, 448), 4),
                          rng.choice(np.arange(448, 4544), 12), rng.choice(np.arange(4544, 4608), 4),
                          rng.choice(np.arange(4608, 4672), 6), [4672]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, norm, X, logT, bf16=False)[0] -
              mlp.loss_and_grad(pm, norm, X, logT, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_rounding():
    # exactly representable values survive; halfway cases round to even
    vals = np.array([1.0, -2.5, 0.15625, 2.0 ** 100, 1.0 + 2 ** -7], dtype=np.float32)
    assert np.array_equal(mlp.bf16_round(vals), vals.astype(np.float64))
    x = np.float32(1.0 + 2 ** -8)  # halfway between 1 and 1 + 2^-7: even mantissa is 1
    assert mlp.bf16_round(x) == 1.0
    y = np.float32(1.0 + 3 * 2 ** -8)  # halfway between 1 + 2^-7 and 1 + 2^-6: round up
    assert mlp.bf16_round(y) == 1.0 + 2 ** -6
    z = np.float32(1.0 + 2 ** -8 + 2 ** -12)  # above halfway: round up
    assert mlp.bf16_round(z) == 1.0 + 2 ** -7


def test_forward_matches_loop():
    p, norm, X, _ = _setup(2, 5)
    y, _ = mlp.forward(p, norm, X, bf16=False)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    for k in range(5):
        x = (X[k] - norm[:6]) / norm[6:12]
        h1 = [mlp.silu(sum(W1[j, i] * x[i] for i in range(6)) + b1[j]) for j in range(64)]
        h2 = [mlp.silu(sum(W2[j, i] * h1[i] for i in range(64)) + b2[j]) for j in range(64)]
        ref = sum(W3[j] * h2[j] for j in range(64)) + b3
        assert abs(ref - y[k]) < 1e-12
