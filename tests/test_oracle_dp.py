"""Pins of the oracle's UC dynamic program (Algorithm 2) against brute force.

The brute force (oracle/bruteforce.py) enumerates schedules, checks Eq. set:UC
as written and evaluates the UC objective in its original (y, z, ubar) form,
so a wrong target formula, a dropped cost term or a wrong hold rule in the DP
changes its argmin and fails these tests.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "uc_dp_cases.json")


def _case(rng, T):
    TU = int(rng.integers(1, min(T, 4) + 1))
    TD = int(rng.integers(1, min(T, 4) + 1))
    u0 = int(rng.integers(0, 2))
    K0 = int(rng.integers(0, 3))
    L, F = (K0, 0) if u0 else (0, K0)
    c0, csu, csd = rng.uniform(0, 400), rng.uniform(0, 900), rng.uniform(0, 300)
    rho = float(rng.choice([1e2, 1e3, 1e4]))
    ubar = rng.uniform(0, 1, (3, T))
    y = rng.normal(0, 0.3 * rho, (3, T))
    z = rng.normal(0, 0.05, (3, T))
    return dict(T=T, TU=TU, TD=TD, u0=u0, K0=K0, L=L, F=F, c0=c0, csu=csu, csd=csd, rho=rho, ubar=ubar, y=y, z=z)


def _dp(c):
    rho = c["rho"]
    tau = (c["ubar"] - c["z"]) - c["y"] / rho
    Lt = oracle.uc_stagecost(c["c0"], c["csu"], c["csd"], rho, tau[0], tau[1], tau[2])
    cost, u = oracle.dp(Lt, c["TU"], c["TD"], c["u0"], c["K0"])
    return cost, u


@pytest.mark.parametrize("seed", range(40))
def test_dp_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    c = _case(rng, int(rng.integers(2, 11)))
    cost, u = _dp(c)
    args = (c["u0"], c["c0"], c["csu"], c["csd"], c["rho"], c["ubar"], c["y"], c["z"])
    assert bf.feasible(u, c["u0"], c["L"], c["F"], c["TU"], c["TD"])
    fbest, ubest = bf.best_schedule(c["T"], c["u0"], c["L"], c["F"], c["TU"], c["TD"], *args[1:])
    fdp = bf.objective(u, *args)
    assert fdp <= fbest + 1e-12 * max(1.0, abs(fbest)), (fdp, fbest, u, ubest)
    # the DP value equals the objective of its schedule up to the constant dropped by the target form
    const = -np.sum(c["y"] ** 2) / (2 * c["rho"])
    assert abs(cost + const - fdp) <= 1e-9 * max(1.0, abs(fdp))


def test_dp_joint_bruteforce_is_separable():
    """All 2^(G T) joint schedules of G = 3 generators, T = 6 (Eq. set:UC is
    separable by generator, Sec. II-B)."""
    rng = np.random.default_rng(7)
    cases = [_case(rng, 6) for _ in range(3)]
    per = []
    for c in cases:
        per.append([(bf.objective(np.array(b), c["u0"], c["c0"], c["csu"], c["csd"], c["rho"], c["ubar"], c["y"],
                                  c["z"]) if bf.feasible(np.array(b), c["u0"], c["L"], c["F"], c["TU"], c["TD"])
                     else np.inf) for b in np.ndindex(*(2,) * 6)])
    per = [np.array(p) for p in per]
    joint = (per[0][:, None, None] + per[1][None, :, None] + per[2][None, None, :]).min()
    assert per[0].size * per[1].size * per[2].size == 2 ** 18
    dp_total = 0.0
    for c in cases:
        _, u = _dp(c)
        dp_total += bf.objective(u, c["u0"], c["c0"], c["csu"], c["csd"], c["rho"], c["ubar"], c["y"], c["z"])
    assert abs(dp_total - joint) <= 1e-12 * abs(joint)


def test_min_time_one_reduces_to_two_state_viterbi():
    rng = np.random.default_rng(3)
    for _ in range(20):
        T = int(rng.integers(1, 30))
        Lt = rng.normal(0, 100, (T, 4))
        u0 = int(rng.integers(0, 2))
        cost, u = oracle.dp(Lt, 1, 1, u0, 0)
        # textbook Viterbi over states {0,1} with transition cost L_t(a,b)
        V = np.array([np.inf, np.inf])
        V[u0] = 0.0
        for t in range(T):
            V = np.array([min(V[a] + Lt[t, a * 2 + b] for a in (0, 1)) for b in (0, 1)])
        assert abs(cost - V.min()) <= 1e-9 * max(1, abs(V.min()))
        path = sum(Lt[t, (u0 if t == 0 else u[t - 1]) * 2 + u[t]] for t in range(T))
        assert abs(path - cost) <= 1e-9 * max(1, abs(cost))


def test_switching_cost_dominates_means_stay():
    T = 12
    for u0 in (0, 1):
        Lt = np.zeros((T, 4))
        Lt[:, 1] = 1e9  # start-up
        Lt[:, 2] = 1e9  # shut-down
        Lt[:, 0] = 5.0
        Lt[:, 3] = 1.0
        _, u = oracle.dp(Lt, 2, 2, u0, 0)
        assert np.all(u == u0)


def test_tie_rule_prefers_stay():
    # every schedule costs 0: Algorithm 2 stays (c_stay <= c_switch)
    Lt = np.zeros((8, 4))
    for u0 in (0, 1):
        c, u = oracle.dp(Lt, 3, 2, u0, 0)
        assert c == 0.0 and np.all(u == u0)


def test_forced_initial_periods():
    T = 8
    Lt = np.zeros((T, 4))
    Lt[:, 3] = 10.0  # being on is expensive
    _, u = oracle.dp(Lt, 1, 1, 1, 3)
    assert np.all(u[:3] == 1) and np.all(u[3:] == 0)


def test_golden_cases():
    """Stored optimal costs of fixed cases, written by tests/golden/make_golden.py
    from the brute-force enumerator."""
    cases = json.load(open(GOLD))
    assert len(cases) >= 10
    for c in cases:
        for k in ("ubar", "y", "z"):
            c[k] = np.array(c[k])
        _, u = _dp(c)
        f = bf.objective(u, c["u0"], c["c0"], c["csu"], c["csd"], c["rho"], c["ubar"], c["y"], c["z"])
        assert abs(f - c["best"]) <= 1e-9 * max(1.0, abs(c["best"])), c["name"]
        assert list(u) == c["schedule"] or abs(f - c["best"]) <= 1e-12 * abs(c["best"])


def test_batched_dp_equals_per_generator_dp():
    rng = np.random.default_rng(11)
    T, ng = 24, 40
    tau = [rng.uniform(-0.3, 1.3, (T, ng)) for _ in range(3)]
    c0, csu, csd = rng.uniform(0, 500, ng), rng.uniform(0, 900, ng), rng.uniform(0, 100, ng)
    TU, TD = rng.integers(1, 6, ng), rng.integers(1, 6, ng)
    u0, K0 = rng.integers(0, 2, ng), rng.integers(0, 3, ng)
    u, cost = oracle.ucdp_batch(1e3, *tau, c0, csu, csd, TU, TD, u0, K0)
    for g in range(ng):
        L = oracle.uc_stagecost(c0[g], csu[g], csd[g], 1e3, tau[0][:, g], tau[1][:, g], tau[2][:, g])
        c, ug = oracle.dp(L, TU[g], TD[g], u0[g], K0[g])
        assert c == cost[g] and np.array_equal(ug, u[:, g])
