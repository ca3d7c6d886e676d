"""UC warm start (Sec. IV-A): relaxed sweeps in lockstep with the oracle,
and the whole procedure -- relaxed sweeps, marks from the generation
levels, the Algorithm-2 repair, the restart from the cold start -- against
the same steps run by the oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_13145_b300 import synth
from tests._helpers import compare_states
from tests.test_gpu_parity import POLAR_SKIP

pytestmark = pytest.mark.gpu


def test_relaxed_uc_lockstep(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    p = ucac_mod.ucac_default_params(uc_relax=1)
    h = ucac_mod.Handle([g], params=p)
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, uc_relax=1))
    for s in range(25):
        pre = h.export(0)
        h.enqueue(1)
        o.set_state(pre)
        o.sweep()
        bad = compare_states(h.export(0), o.state_vector(), g, skip=POLAR_SKIP, mu_eta=p.eta)
        assert not bad, f"sweep {s}: {bad[:6]}"
    st = oracle.unpack_state(h.export(0), g.T, g.n_gen, g.n_branch, g.n_bus)
    assert np.any((st["u_on"] > 0.0) & (st["u_on"] < 1.0)) or np.all(np.isin(st["u_on"], (0.0, 1.0)))
    h.close()


def _oracle_warm_start(g, cold, sweeps, p_frac):
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, uc_relax=1))
    o.set_state(cold)
    o.sweep(sweeps)
    st = oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
    sched = np.zeros((g.T, g.n_gen))
    for k in range(g.n_gen):
        m = (st["p"][:, k] >= p_frac * g.Pmin[k]).astype(float)
        prev = np.concatenate([[float(g.u0[k])], m[:-1]])
        su, sd = (m > prev).astype(float), (prev > m).astype(float)
        L = oracle.uc_stagecost(0.0, 0.0, 0.0, 1.0, m, su, sd)
        K0 = int(g.L0[k] if g.u0[k] else g.F0[k])
        _, u = oracle.dp(L, max(int(g.TU[k]), 1), max(int(g.TD[k]), 1), int(g.u0[k]), min(K0, g.T))
        sched[:, k] = u
    return sched


@pytest.mark.parametrize("name,sweeps", [("c1_9bus_T6", 120), ("c2_118bus_T24x3", 60)])
def test_uc_warm_start_matches_oracle(ucac_mod, name, sweeps):
    g = synth.config_instances(name)[0]
    h = ucac_mod.Handle([g])
    cold = h.export(0)
    h.uc_warm_start(sweeps, 0.5)
    after = oracle.unpack_state(h.export(0), g.T, g.n_gen, g.n_branch, g.n_bus)
    sched = _oracle_warm_start(g, cold, sweeps, 0.5)
    assert np.array_equal(after["u_on"], sched)
    assert np.array_equal(after["ub_on"], sched)
    prev = np.concatenate([g.u0[None, :].astype(float), sched[:-1]], 0)
    assert np.array_equal(after["u_su"], (sched > prev).astype(float))
    assert np.array_equal(after["u_sd"], (prev > sched).astype(float))
    # everything else is the cold start again
    c = oracle.unpack_state(cold, g.T, g.n_gen, g.n_branch, g.n_bus)
    for name_, v in c.items():
        if name_ in ("u_on", "u_su", "u_sd", "ub_on", "ub_su", "ub_sd"):
            continue
        assert np.array_equal(np.asarray(after[name_]), np.asarray(v)), name_
    assert h.residuals(0)["sweeps"] == 0
    # the restarted method runs and the schedule is a real decision
    h.enqueue(50)
    assert np.isfinite(h.residuals(0)["r_p"])
    h.close()
