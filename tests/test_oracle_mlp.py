"""Pins of the FP64 warm-start network reference (oracle/mlp.py).

The backpropagation is checked against central finite differences of the
loss (a plausible slip -- a transposed weight, a dropped SiLU derivative
term, a wrong 1/n -- fails it); the BF16 rounding against values whose
rounding is fixed by the format; the BF16 forward against the FP64 forward.
"""
import numpy as np

from oracle import mlp


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(seed=1).astype(np.float64) + rng.normal(0, 0.05, mlp.NPARAM)
    X = rng.normal(0, 1, (7, mlp.IN))
    L = rng.normal(0, 1, (7, mlp.OUT))
    _, g = mlp.loss_grad(p, X, L)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False),
                          [0, 767, 768, 831, 832, 4927, 4928, 4991, 4992, 5375, 5376, 5381]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_grad(p + e, X, L)[0] - mlp.loss_grad(p - e, X, L)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_mean_squared_error_of_forward():
    rng = np.random.default_rng(2)
    p = mlp.init_params(seed=3)
    X = rng.normal(0, 1, (11, mlp.IN))
    L = rng.normal(0, 1, (11, mlp.OUT))
    loss, _ = mlp.loss_grad(p, X, L)
    assert abs(loss - np.sum((mlp.forward(p, X) - L) ** 2) / 11) <= 1e-12 * loss


def test_param_count_and_layout():
    assert mlp.NPARAM == 64 * 12 + 64 + 64 * 64 + 64 + 6 * 64 + 6 == 5382
    P = mlp.unpack(np.arange(mlp.NPARAM, dtype=np.float64))
    assert P["W1"][1, 0] == 12 and P["b1"][0] == 768 and P["W2"][0, 1] == 833 and P["b3"][5] == 5381


def test_bf16_rounding():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)  # BF16 spacing at 1
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5, 0.0],
                    np.float32)
    r = mlp.to_bf16(vals)
    # halfway cases round to even: 1 + ulp/2 -> 1, 1 + 3 ulp/2 -> 1 + 2 ulp
    assert r[0] == one and r[1] == one and r[2] == one + 2 * ulp and r[3] == one + ulp
    assert r[4] == np.float32(-2.5) and r[5] == 0.0


def test_bf16_forward_close_to_fp64():
    rng = np.random.default_rng(4)
    p = mlp.init_params(seed=5)
    X = rng.normal(0, 1, (256, mlp.IN))
    y64, y16 = mlp.forward(p, X), mlp.forward_bf16(p, X)
    assert np.max(np.abs(y16 - y64)) <= 0.05 * max(1.0, np.max(np.abs(y64)))
    assert np.max(np.abs(y16 - y64)) > 0  # the rounding is really applied
