"""FP64 reference of the learned warm start: network, loss gradient, features.

TEST INFRASTRUCTURE ONLY (same rule as the rest of this package): the tests
and the benchmark's CPU legs may use it; the library never does, and nothing
here calls the library.

The network is 12 -> 64 -> 64 -> 6 with SiLU activations, parameters in one
flat vector W1 [64][12], b1 [64], W2 [64][64], b2 [64], W3 [6][64], b3 [6].
`loss_grad` is written-out backpropagation of L = (1/n) sum |y - label|^2;
it is pinned by central finite differences in the tests.  `forward_bf16`
mimics the tensor-core inference precision (BF16 inputs, weights and hidden
activations, FP32 accumulation and epilogue).  `line_features` is the
definition of the 12 features from a canonical state vector.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 12, 64, 6
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def init_params(seed=0, scale=1.0):
    """He-style random initialisation (as float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SIZES:
        if name.startswith("W"):
            parts.append(rng.normal(0.0, scale * np.sqrt(2.0 / shp[1]), shp).reshape(-1))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts).astype(np.float32)


def silu(z):
    return z / (1.0 + np.exp(-z))


def forward(p, X):
    P = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = silu(X @ P["W1"].T + P["b1"])
    h2 = silu(h1 @ P["W2"].T + P["b2"])
    return h2 @ P["W3"].T + P["b3"]


def loss_grad(p, X, L):
    """(loss, gradient as a flat vector) of (1/n) sum_b |y_b - L_b|^2."""
    P = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    n = X.shape[0]
    z1 = X @ P["W1"].T + P["b1"]
    s1 = 1.0 / (1.0 + np.exp(-z1))
    h1 = z1 * s1
    z2 = h1 @ P["W2"].T + P["b2"]
    s2 = 1.0 / (1.0 + np.exp(-z2))
    h2 = z2 * s2
    y = h2 @ P["W3"].T + P["b3"]
    e = y - L
    loss = float(np.sum(e * e) / n)
    dy = 2.0 * e / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ P["W3"]) * (s2 * (1.0 + z2 * (1.0 - s2)))
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (s1 * (1.0 + z1 * (1.0 - s1)))
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, np.concatenate([g[name].reshape(-1) for name, _ in SIZES])


def to_bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def forward_bf16(p, X):
    """Inference in the tensor-core precision: BF16 operands, FP32 sums."""
    P = {k: v.astype(np.float32) for k, v in unpack(p).items()}
    x = to_bf16(X)
    z1 = x @ to_bf16(P["W1"]).T + P["b1"]
    h1 = to_bf16(z1 / (1.0 + np.exp(-z1)))
    z2 = h1 @ to_bf16(P["W2"]).T + P["b2"]
    h2 = to_bf16(z2 / (1.0 + np.exp(-z2)))
    return h2 @ to_bf16(P["W3"]).T + P["b3"]


def line_features(st, grid, T, rho_pq, rho_va):
    """Features [T*n_branch][12] and residual norms |r| of a canonical state
    (dict from oracle.unpack_state): see the feature list in the module doc
    of the CUDA kernel; targets t = (x-bar - z) - y / rho of the line rows."""
    nl = grid.n_branch
    fb = [st["fb%d" % k] for k in range(4)]
    wbar, thbar = st["wbar"], st["thbar"]
    i, j = np.asarray(grid.br_from), np.asarray(grid.br_to)
    bv = fb + [wbar[:, i], wbar[:, j], thbar[:, i], thbar[:, j]]
    tg = []
    for r, name in enumerate(["pij", "qij", "pji", "qji", "wi", "wj", "thi", "thj"]):
        rho = rho_pq if r < 4 else rho_va
        tg.append((bv[r] - st["bz_" + name]) - st["by_" + name] / rho)
    wi, wj, wR, wI, thi, thj = (st["v%d" % k] for k in range(6))
    r_, x_ = np.asarray(grid.br_r), np.asarray(grid.br_x)
    z2 = r_ * r_ + x_ * x_
    gs, bs = r_ / z2, -x_ / z2
    bc = np.asarray(grid.br_b)
    Gii, Bii, Gij, Bij = gs, bs + 0.5 * bc, -gs, -bs
    Gjj, Bjj, Gji, Bji = gs, bs + 0.5 * bc, -gs, -bs
    a = [Gii * wi + Gij * wR + Bij * wI, -Bii * wi - Bij * wR + Gij * wI,
         Gjj * wj + Gji * wR - Bji * wI, -Bjj * wj - Bji * wR - Gji * wI]
    ym = np.sqrt(gs * gs + bs * bs)
    res = [(tg[r] - a[r]) / ym for r in range(4)] + [tg[4] - wi, tg[5] - wj, (tg[6] - tg[7]) - (thi - thj)]
    res = np.stack(res, -1).reshape(T * nl, 7)
    s = np.sqrt(np.sum(res * res, -1))
    base = np.stack([np.sqrt(np.maximum(wi, 0.0)), np.sqrt(np.maximum(wj, 0.0)), thi - thj,
                     np.broadcast_to(gs / ym, wi.shape), np.broadcast_to(bs / ym, wi.shape)], -1).reshape(T * nl, 5)
    unit = np.where(s[:, None] > 1e-300, res / np.where(s > 1e-300, s, 1.0)[:, None], 0.0)
    return np.concatenate([base, unit], 1), s
