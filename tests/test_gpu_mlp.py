"""Learned warm start on the GPU: tensor-core inference, training kernels,
features, and the solver with the network switched on.

Inference is compared with the FP64 reference run in the kernel's own
precision (BF16 operands and hidden activations, FP32 sums); the FP32
training gradient with the FP64 backpropagation of the oracle; the feature
kernel with the feature definition evaluated on the exported state.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2310_13145_b300 import synth, warmstart
from tests._helpers import compare_states
from tests.test_gpu_parity import POLAR_SKIP, _lockstep

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 70001])
def test_tensor_core_forward_matches_bf16_reference(ucac_mod, n):
    rng = np.random.default_rng(n)
    p = mlp.init_params(seed=7)
    p[mlp.NPARAM - 6:] = rng.normal(0, 0.1, 6)  # non-zero output bias
    p[768:832] = rng.normal(0, 0.1, 64)
    X = rng.normal(0, 1, (n, mlp.IN)).astype(np.float32)
    y = warmstart.predict(p, X)
    ref = mlp.forward_bf16(p, X)
    err = np.abs(y - ref)
    scale = max(1.0, float(np.max(np.abs(ref))))
    # identical rounding points; differences come from the FP32 summation
    # order and exp, which can flip a BF16 rounding of a hidden activation
    assert float(np.max(err)) <= 2e-2 * scale, float(np.max(err))
    assert float(np.median(err)) <= 1e-3 * scale


def test_tensor_core_forward_is_not_trivial(ucac_mod):
    """A wrong operand layout would still give finite numbers: check that
    every output column follows its own weights."""
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (256, mlp.IN)).astype(np.float32)
    p = mlp.init_params(seed=2)
    y0 = warmstart.predict(p, X)
    for j in range(mlp.OUT):
        q = p.copy()
        q[4992 + 64 * j:4992 + 64 * (j + 1)] *= 2.0  # W3 row j
        q[5376 + j] += 1.0
        y1 = warmstart.predict(q, X)
        other = [c for c in range(mlp.OUT) if c != j]
        assert np.allclose(y1[:, other], y0[:, other])
        assert np.allclose(y1[:, j], 2.0 * (y0[:, j] - p[5376 + j]) + p[5376 + j] + 1.0, atol=2e-2)


def test_training_gradient_matches_oracle(ucac_mod):
    rng = np.random.default_rng(3)
    p = mlp.init_params(seed=4) + rng.normal(0, 0.02, mlp.NPARAM).astype(np.float32)
    X = rng.normal(0, 1, (1000, mlp.IN)).astype(np.float32)
    L = rng.normal(0, 1, (1000, mlp.OUT)).astype(np.float32)
    tr = warmstart.Trainer(p, batch=1000)
    g, loss = tr.grad(torch.tensor(X, device="cuda"), torch.tensor(L, device="cuda"))
    lo, go = mlp.loss_grad(p.astype(np.float64), X, L)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go)
    for name, (a, b) in {"W1": (0, 768), "b1": (768, 832), "W2": (832, 4928), "b2": (4928, 4992),
                         "W3": (4992, 5376), "b3": (5376, 5382)}.items():
        assert np.linalg.norm(gg[a:b] - go[a:b]) <= 1e-4 * max(np.linalg.norm(go[a:b]), 1e-12), name


def test_adam_step(ucac_mod):
    rng = np.random.default_rng(5)
    p = rng.normal(0, 1, mlp.NPARAM).astype(np.float32)
    g = rng.normal(0, 1, mlp.NPARAM).astype(np.float32)
    m = rng.normal(0, 0.1, mlp.NPARAM).astype(np.float32)
    v = np.abs(rng.normal(0, 0.1, mlp.NPARAM)).astype(np.float32)
    t = {k: torch.tensor(a, device="cuda") for k, a in (("p", p), ("g", g), ("m", m), ("v", v))}
    ucac_mod.ucac_mlp_adam(t["p"].data_ptr(), t["g"].data_ptr(), t["m"].data_ptr(), t["v"].data_ptr(), 3, 1e-3,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    m, v, g, p = (a.astype(np.float64) for a in (m, v, g, p))
    m1 = 0.9 * m + 0.1 * g
    v1 = 0.999 * v + 0.001 * g * g
    p1 = p - 1e-3 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    # FP32 kernel against the FP64 formula: a few FP32 roundings apart
    assert np.allclose(t["m"].cpu().numpy(), m1, rtol=1e-6, atol=1e-7)
    assert np.allclose(t["v"].cpu().numpy(), v1, rtol=1e-5, atol=1e-8)
    assert np.allclose(t["p"].cpu().numpy(), p1, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("name", ["c1_9bus_T6", "c2_118bus_T24x3"])
def test_line_features_match_definition(ucac_mod, name):
    g = synth.config_instances(name)[0]
    h = ucac_mod.Handle([g])
    h.enqueue(7)
    f, s = h.line_features(0)
    st = oracle.unpack_state(h.export(0), g.T, g.n_gen, g.n_branch, g.n_bus)
    fo, so = mlp.line_features(st, g, g.T, g.rho[0], g.rho[1])
    assert np.allclose(s, so, rtol=1e-9, atol=1e-300)
    assert np.max(np.abs(f - fo)) <= 1e-6 * max(1.0, float(np.max(np.abs(fo))))
    h.close()


def test_warm_start_lockstep_parity(ucac_mod):
    """With an (untrained) network proposing the start of every line solve,
    each sweep still matches the oracle's sweep from the same state: the
    Newton solve polishes to the same tolerance whatever its start."""
    g = synth.config_instances("c1_9bus_T6")[0]
    p = mlp.init_params(seed=11, scale=0.3)
    hs = {}

    def setup(h):
        h.set_warm_start(p)
        hs["h"] = h

    _lockstep(ucac_mod, [g], 20, setup=setup, line_form=ucac_mod.UCAC_LINE_POLAR)


def test_trained_warm_start_gain(ucac_mod):
    """Trains the network on line solves logged from 9-bus runs (seeds
    100..), evaluates on a held-out 118-bus instance: the trained network
    predicts the change of the line iterates better than the plain start
    (which predicts no change); over 200 sweeps with it on the line solves
    take fewer Newton iterations than without it, and the run ends at the
    same residuals and objective (the Newton solve polishes either start to
    the same tolerance)."""
    X, Y = [], []
    for seed in range(100, 106):
        g = synth.make_grid(9, 9, 3, 6, seed=seed, load_seed=seed, name="c1_9bus_T6_train%d" % seed)
        h = ucac_mod.Handle([g])
        x, y = warmstart.collect(h, 60)
        X.append(x)
        Y.append(y)
        h.close()
    X, Y = np.concatenate(X), np.concatenate(Y)
    tr = warmstart.Trainer(warmstart.init_params(0), batch=1024, lr=2e-3)
    hist = tr.fit(X, Y, epochs=8)
    assert hist[-1] < hist[0]
    p = tr.params()
    g = synth.config_instances("c2_118bus_T24x3")[2]
    h = ucac_mod.Handle([g])
    h.enqueue(20)
    Xv, Yv = warmstart.collect(h, 10)
    h.close()
    yv = warmstart.predict(p, Xv)
    mse_net = float(np.mean(np.sum((yv - Yv) ** 2, 1)))
    mse_zero = float(np.mean(np.sum(Yv ** 2, 1)))
    print(f"held-out 118-bus: network MSE {mse_net:.4g} vs plain start {mse_zero:.4g}")
    assert mse_net < mse_zero
    runs = {}
    for mode in ("plain", "learned"):
        h = ucac_mod.Handle([g])
        if mode == "learned":
            h.set_warm_start(p)
        newton = 0
        for _ in range(200):
            h.enqueue(1)
            newton += h.residuals(0)["newton"]
        taken, err = h.warm_start_stats(0)
        r = h.residuals(0)
        runs[mode] = (newton, taken, err, r["r_p"], r["objective"])
        h.close()
    print("Newton iterations over 200 sweeps:", runs)
    assert runs["learned"][2] == 0 and runs["learned"][1] > 0
    assert runs["learned"][0] < runs["plain"][0], runs
    assert abs(runs["learned"][3] - runs["plain"][3]) <= 1e-6 * runs["plain"][3]
    assert abs(runs["learned"][4] - runs["plain"][4]) <= 1e-6 * abs(runs["plain"][4])
