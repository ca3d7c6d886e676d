"""Standalone UC dynamic program (Algorithm 2) on the GPU vs the oracle's:
decisions and optimal costs bit for bit, including constructed near-ties."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _run_gpu(ucac, tau_on, tau_su, tau_sd, c0, csu, csd, TU, TD, u0, K0, rho):
    import torch
    T, ng = tau_on.shape
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    A = [t(tau_on, torch.float64), t(tau_su, torch.float64), t(tau_sd, torch.float64), t(c0, torch.float64),
         t(csu, torch.float64), t(csd, torch.float64), t(TU, torch.int32), t(TD, torch.int32), t(u0, torch.int32),
         t(K0, torch.int32)]
    u = torch.zeros((T, ng), dtype=torch.int8, device=dev)
    cost = torch.zeros(ng, dtype=torch.float64, device=dev)
    nbytes = ucac.ucac_ucdp_workspace_bytes(ng, T)
    ws = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    ucac.ucac_ucdp(ng, T, rho, *[a.data_ptr() for a in A], u.data_ptr(), cost.data_ptr(), ws.data_ptr(), nbytes,
                   stream)
    torch.cuda.synchronize()
    return u.cpu().numpy(), cost.cpu().numpy()


# (ucac_ucdp runs a warp per generator up to 2,048 generators, with its
# tables in shared memory -- more than 48 KB of it from T ~ 190 on -- and a
# thread per generator beyond: cases on both sides of each threshold)
@pytest.mark.parametrize("T,ng,seed", [(24, 1000, 0), (1, 7, 1), (2, 33, 2), (168, 257, 3), (48, 10000, 4),
                                       (24, 2048, 5), (24, 2049, 6), (600, 64, 7)])
def test_ucdp_bit_exact(ucac_mod, T, ng, seed):
    rng = np.random.default_rng(seed)
    rho = 1e4
    tau_on = rng.uniform(-0.5, 1.5, (T, ng))
    tau_su = rng.uniform(-0.5, 1.5, (T, ng))
    tau_sd = rng.uniform(-0.5, 1.5, (T, ng))
    c0 = rng.uniform(0, 3000, ng)
    csu = rng.uniform(0, 5000, ng)
    csd = rng.uniform(0, 1000, ng)
    TU = rng.integers(1, 6, ng).astype(np.int32)
    TD = rng.integers(1, 6, ng).astype(np.int32)
    u0 = rng.integers(0, 2, ng).astype(np.int32)
    K0 = rng.integers(0, 3, ng).astype(np.int32)
    # near-ties: make some generators' on/off costs exactly symmetric
    tie = rng.random(ng) < 0.2
    tau_on[:, tie] = 0.5
    c0[tie] = 0.0
    csu[tie] = 0.0
    csd[tie] = 0.0
    tau_su[:, tie] = 0.0
    tau_sd[:, tie] = 0.0
    u, cost = _run_gpu(ucac_mod, tau_on, tau_su, tau_sd, c0, csu, csd, TU, TD, u0, K0, rho)
    for g in range(ng):
        L = oracle.uc_stagecost(c0[g], csu[g], csd[g], rho, tau_on[:, g], tau_su[:, g], tau_sd[:, g])
        c, uo = oracle.dp(L, TU[g], TD[g], u0[g], K0[g])
        assert np.array_equal(uo, u[:, g].astype(np.int32)), g
        assert c == cost[g], (g, c, cost[g])
