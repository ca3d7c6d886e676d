"""Learned warm start of the line subproblems: data collection and training.

Samples come from the method's own runs: before a sweep, the library's
feature kernel gives each line-period's 12 features and residual norm s;
after the sweep, the label is the change of the line's W-form iterate
(w_i, w_j, wR, wI, theta_i, theta_j) divided by s.  Training runs the
library's own FP32 forward/backward kernels and Adam step on the GPU
(PyTorch only holds the device buffers and shuffles the batches); inference
inside the sweep uses the BF16 tensor-core kernel (ucac_set_warm_start).
"""
from __future__ import annotations

import numpy as np
import torch

from . import ucac


def collect(handle: ucac.Handle, n_sweeps: int, stride: int = 1, min_scale: float = 1e-12):
    """Runs n_sweeps sweeps on the handle and returns (X [N][12], Y [N][6])
    float32 from every `stride`-th sweep's line solves of all its instances
    (rows with a residual norm below min_scale are skipped: the solve does
    not move there)."""
    xs, ys = [], []
    for s in range(n_sweeps):
        if s % stride:
            handle.enqueue(1)
            continue
        f, sc, x0 = handle.line_samples()
        handle.enqueue(1)
        _, _, x1 = handle.line_samples(features=False)
        keep = sc > min_scale
        xs.append(f[keep])
        ys.append(((x1[keep] - x0[keep]) / sc[keep, None]).astype(np.float32))
    return np.concatenate(xs), np.concatenate(ys)


def train_default(n_instances: int = 100, sweeps: int = 300, stride: int = 2, epochs: int = 6, batch: int = 4096,
                  lr: float = 2e-3, seed: int = 0):
    """The default network: trained on line solves logged from runs of
    9-bus grids (T = 6, seeds 100, 101, ...; all instances batched in one
    handle).  Returns (params, info)."""
    from . import synth
    grids = [synth.make_grid(9, 9, 3, 6, seed=100 + i, load_seed=100 + i, name="c1_9bus_T6_train%d" % i)
             for i in range(n_instances)]
    h = ucac.Handle(grids)
    X, Y = collect(h, sweeps, stride)
    h.close()
    tr = Trainer(init_params(seed), batch=batch, lr=lr)
    hist = tr.fit(X, Y, epochs=epochs, seed=seed)
    return tr.params(), {"samples": int(X.shape[0]), "epochs": epochs, "loss_first": hist[0], "loss_last": hist[-1],
                         "train_grids": "%d x 9-bus T=6 (seeds 100..%d)" % (n_instances, 99 + n_instances)}


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation of the flat parameter vector (float32)."""
    rng = np.random.default_rng(seed)
    shapes = [(64, 12), (64,), (64, 64), (64,), (6, 64), (6,)]
    parts = [rng.normal(0.0, np.sqrt(2.0 / s[1]), s).ravel() if len(s) == 2 else np.zeros(s) for s in shapes]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ucac.ucac_mlp_param_count()
    return p


class Trainer:
    """Adam on the library's FP32 training kernels; buffers live on the GPU."""

    def __init__(self, params: np.ndarray, batch: int = 4096, lr: float = 1e-3, device="cuda"):
        self.dev = torch.device(device)
        self.p = torch.tensor(params, dtype=torch.float32, device=self.dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.batch = batch
        self.lr = lr
        self.step = 0
        self.ws_bytes = ucac.ucac_mlp_workspace_bytes(batch)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.dev)

    def _stream(self):
        return torch.cuda.current_stream(self.dev).cuda_stream

    def grad(self, xb: torch.Tensor, yb: torch.Tensor):
        n = xb.shape[0]
        ws_bytes = ucac.ucac_mlp_workspace_bytes(n)
        ws = self.ws if ws_bytes <= self.ws_bytes else torch.empty(ws_bytes, dtype=torch.uint8, device=self.dev)
        ucac.ucac_mlp_grad(n, self.p.data_ptr(), xb.data_ptr(), yb.data_ptr(), self.g.data_ptr(),
                           self.loss.data_ptr(), ws.data_ptr(), max(ws_bytes, ws.numel()), self._stream())
        return self.g, self.loss

    def fit(self, X: np.ndarray, Y: np.ndarray, epochs: int = 5, seed: int = 0) -> list:
        Xd = torch.tensor(X, dtype=torch.float32, device=self.dev)
        Yd = torch.tensor(Y, dtype=torch.float32, device=self.dev)
        gen = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        n = Xd.shape[0]
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen).to(self.dev)
            tot, nb = 0.0, 0
            for b in range(0, n - self.batch + 1, self.batch):
                idx = perm[b:b + self.batch]
                xb, yb = Xd[idx].contiguous(), Yd[idx].contiguous()
                self.grad(xb, yb)
                self.step += 1
                ucac.ucac_mlp_adam(self.p.data_ptr(), self.g.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                   self.step, self.lr, self._stream())
                tot += float(self.loss.item())
                nb += 1
            hist.append(tot / max(nb, 1))
        return hist

    def params(self) -> np.ndarray:
        return self.p.detach().cpu().numpy().copy()


def predict(params: np.ndarray, X: np.ndarray, device="cuda") -> np.ndarray:
    """Tensor-core inference (BF16 operands, FP32 accumulation) of X [n][12]."""
    dev = torch.device(device)
    n = X.shape[0]
    p = torch.tensor(params, dtype=torch.float32, device=dev)
    x = torch.tensor(X, dtype=torch.float32, device=dev)
    y = torch.empty((n, 6), dtype=torch.float32, device=dev)
    wb = ucac.ucac_mlp_workspace_bytes(n)
    ws = torch.empty(wb, dtype=torch.uint8, device=dev)
    ucac.ucac_mlp_forward(n, p.data_ptr(), x.data_ptr(), y.data_ptr(), ws.data_ptr(), wb,
                          torch.cuda.current_stream(dev).cuda_stream)
    return y.cpu().numpy()
