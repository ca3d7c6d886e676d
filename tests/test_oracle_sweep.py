"""Instance-level pins of one oracle sweep (Eq. step:uc .. step:y).

Row values are rebuilt here from the iterate, from the coupling rows of
Eq. uc_duplicate .. ramp_up (ramp-down as in Eq. uc_acopf_gen_ramp_down_ineq)
and the consensus rows, and each x-bar step is re-solved by a generic method:
  - x-bar^UC over all 3T duplicate variables of a generator at once (bounded
    least squares), which checks the block separation of reading R7;
  - each bus by a dense KKT solve of the balance-constrained QP (R8);
  - z and y by their optimality / update equations (R9, R10);
  - residuals in long double (R11);
  - the x^UC step by brute force over all schedules (Algorithm 2).
"""
import numpy as np
import pytest
from scipy.optimize import lsq_linear

import oracle
from oracle import bruteforce as bf
from paper_2310_13145_b300 import synth

GR = {r: i for i, r in enumerate(oracle.GEN_ROWS)}
BR = {r: i for i, r in enumerate(oracle.BR_ROWS)}


@pytest.fixture(scope="module", params=[False, True], ids=["plain", "shunts"])
def swept(request):
    # the second grid adds bus shunts (coupled P/Q balance multipliers) and
    # line charging
    g = synth.config_instances("c1_9bus_T6", shunts=request.param)[0]
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, L_max=5))
    o.sweep(27)
    pre = o.state()
    pre_vec = o.state_vector()
    o.sweep()
    post = o.state()
    GA, GB, BA, BB = o.rows()
    return g, o, pre, pre_vec, post, GA, GB, BA, BB


def _rho_g(g, r):
    return g.rho[2] if r in ("on", "su", "sd") else g.rho[0]


def test_xbar_uc_solves_joint_problem(swept):
    g, o, pre, _, post, GA, GB, BA, BB = swept
    T = g.T
    for gi in range(g.n_gen):
        rows, rhs, w = [], [], []

        def add(coef, const, r, t):
            rho = _rho_g(g, r)
            m = GA[GR[r], t, gi] + pre["gz_" + r][t, gi] + pre["gy_" + r][t, gi] / rho
            rows.append(np.sqrt(rho) * coef)
            rhs.append(np.sqrt(rho) * (m - const))

        n = 3 * T  # variables: on[0..T), su[0..T), sd[0..T)
        for t in range(T):
            e = lambda k, tt: np.eye(n)[k * T + tt]
            add(e(0, t), 0.0, "on", t)
            add(e(1, t), 0.0, "su", t)
            add(e(2, t), 0.0, "sd", t)
            add(g.Pmin[gi] * e(0, t), 0.0, "pl", t)
            add(g.Pmax[gi] * e(0, t), 0.0, "pu", t)
            add(g.Qmin[gi] * e(0, t), 0.0, "ql", t)
            add(g.Qmax[gi] * e(0, t), 0.0, "qu", t)
            add(-g.RD[gi] * e(0, t) - g.SD[gi] * e(2, t), 0.0, "rd", t)
            if t == 0:
                add(g.SU[gi] * e(1, 0), g.RU[gi] * g.u0[gi], "ru", 0)
            else:
                add(g.RU[gi] * e(0, t - 1) + g.SU[gi] * e(1, t), 0.0, "ru", t)
        ref = lsq_linear(np.array(rows), np.array(rhs), bounds=(0, 1), method="bvls", tol=1e-15).x
        got = np.concatenate([post["ub_on"][:, gi], post["ub_su"][:, gi], post["ub_sd"][:, gi]])
        assert np.allclose(got, ref, atol=1e-9), (gi, got - ref)


def test_bus_steps_solve_dense_kkt(swept):
    g, o, pre, _, post, GA, GB, BA, BB = swept
    rpq, rva, _ = g.rho
    T = g.T
    mt = lambda a, z, y, rho: a + z + y / rho
    for t in range(T):
        for i in range(g.n_bus):
            W, m, aP, aQ, got = [], [], [], [], []
            for gi in np.nonzero(g.gen_bus == i)[0]:
                ms = [mt(GA[GR["gp"], t, gi], pre["gz_gp"][t, gi], pre["gy_gp"][t, gi], rpq)]
                if t < T - 1:
                    ms.append(mt(GA[GR["tc"], t + 1, gi], pre["gz_tc"][t + 1, gi], pre["gy_tc"][t + 1, gi], rpq))
                W.append(rpq * len(ms)); m.append(np.mean(ms)); aP.append(1.0); aQ.append(0.0)
                got.append(post["pbar"][t, gi])
                W.append(rpq); m.append(mt(GA[GR["gq"], t, gi], pre["gz_gq"][t, gi], pre["gy_gq"][t, gi], rpq))
                aP.append(0.0); aQ.append(1.0); got.append(post["qbar"][t, gi])
            mw, mth, deg = [], [], 0
            for l in range(g.n_branch):
                for side, bus in ((0, g.br_from[l]), (1, g.br_to[l])):
                    if bus != i:
                        continue
                    deg += 1
                    rp, rq = ("pij", "qij") if side == 0 else ("pji", "qji")
                    for r, cp, cq in ((rp, -1.0, 0.0), (rq, 0.0, -1.0)):
                        W.append(rpq); m.append(mt(BA[BR[r], t, l], pre["bz_" + r][t, l], pre["by_" + r][t, l], rpq))
                        aP.append(cp); aQ.append(cq)
                        got.append(post["fb%d" % BR[r]][t, l])
                    rw, rt = ("wi", "thi") if side == 0 else ("wj", "thj")
                    mw.append(mt(BA[BR[rw], t, l], pre["bz_" + rw][t, l], pre["by_" + rw][t, l], rva))
                    mth.append(mt(BA[BR[rt], t, l], pre["bz_" + rt][t, l], pre["by_" + rt][t, l], rva))
            W.append(rva * deg); m.append(np.mean(mw)); aP.append(-g.Gs[i]); aQ.append(g.Bs[i])
            got.append(post["wbar"][t, i])
            n = len(W)
            K = np.zeros((n + 2, n + 2))
            K[:n, :n] = np.diag(W)
            K[:n, n] = K[n, :n] = aP
            K[:n, n + 1] = K[n + 1, :n] = aQ
            sol = np.linalg.solve(K, np.concatenate([np.array(W) * np.array(m), [g.Pd[t, i], g.Qd[t, i]]]))[:n]
            assert np.allclose(got, sol, rtol=1e-11, atol=1e-12), (t, i)
            th = 0.0 if i == g.ref_bus else np.mean(mth)
            assert abs(post["thbar"][t, i] - th) <= 1e-12


def test_z_and_y_updates(swept):
    g, o, pre, _, post, GA, GB, BA, BB = swept
    beta = post["beta"]
    for fam, A, B, rows in (("g", GA, GB, oracle.GEN_ROWS), ("b", BA, BB, oracle.BR_ROWS)):
        for k, r in enumerate(rows):
            if fam == "g":
                rho = _rho_g(g, r)
            else:
                rho = g.rho[0] if r in ("pij", "qij", "pji", "qji") else g.rho[1]
            c = A[k] - B[k]
            z, lam, y0 = post["%sz_%s" % (fam, r)], post["%slam_%s" % (fam, r)], pre["%sy_%s" % (fam, r)]
            mask = np.ones_like(c, bool)
            if r == "tc":
                mask[0] = False
            # d/dz [lam z + beta/2 z^2 + y (c+z) + rho/2 (c+z)^2] = 0
            dz = lam + beta * z + y0 + rho * (c + z)
            assert np.abs(dz[mask]).max() <= 1e-9 * max(1.0, np.abs(lam).max() + np.abs(y0).max() + rho)
            y1 = post["%sy_%s" % (fam, r)]
            assert np.allclose(y1[mask], (y0 + rho * (c + z))[mask], rtol=1e-13, atol=1e-10 * rho)


def test_residuals_recomputed_in_long_double(swept):
    g, o, pre, _, post, GA, GB, BA, BB = swept
    _, _, _, _ = GA, GB, BA, BB
    o2 = oracle.Oracle(g, oracle.default_params(rho=g.rho, L_max=5))
    o2.set_state(pre)
    GB0 = o2.rows()[1]
    BB0 = o2.rows()[3]
    sp = sd = sz = np.longdouble(0)
    m = 0
    inf = 0.0
    for A, B, B0, fam, rows in ((GA, GB, GB0, "g", oracle.GEN_ROWS), (BA, BB, BB0, "b", oracle.BR_ROWS)):
        for k, r in enumerate(rows):
            mask = np.ones(A[k].shape, bool)
            if r == "tc":
                mask[0] = False
            c = (A[k] - B[k])[mask].astype(np.longdouble)
            z = post["%sz_%s" % (fam, r)][mask].astype(np.longdouble)
            sp += np.sum((c + z) ** 2)
            sd += np.sum((B[k][mask].astype(np.longdouble) - B0[k][mask]) ** 2)
            sz += np.sum(z ** 2)
            inf = max(inf, float(np.abs(c).max()))
            m += int(mask.sum())
    res = o.residuals()
    assert m == g.T * 8 * g.n_branch + g.n_gen * (12 * g.T - 1)
    assert abs(res["r_p"] - float(np.sqrt(sp / m))) <= 1e-13 * res["r_p"]
    assert abs(res["r_d"] - float(np.sqrt(sd / m))) <= 1e-13 * res["r_d"]
    assert abs(res["z_norm"] - float(np.sqrt(sz))) <= 1e-13 * res["z_norm"]
    assert res["inf_norm"] == inf


def test_uc_step_is_bruteforce_optimal(swept):
    g, o, pre, _, post, GA, GB, BA, BB = swept
    rho = g.rho[2]
    for gi in range(g.n_gen):
        ubar = np.stack([pre["ub_on"][:, gi], pre["ub_su"][:, gi], pre["ub_sd"][:, gi]])
        y = np.stack([pre["gy_on"][:, gi], pre["gy_su"][:, gi], pre["gy_sd"][:, gi]])
        z = np.stack([pre["gz_on"][:, gi], pre["gz_su"][:, gi], pre["gz_sd"][:, gi]])
        best, _ = bf.best_schedule(g.T, int(g.u0[gi]), int(g.L0[gi]), int(g.F0[gi]), int(g.TU[gi]), int(g.TD[gi]),
                                   g.c0[gi], g.c_su[gi], g.c_sd[gi], rho, ubar, y, z)
        u = post["u_on"][:, gi].astype(int)
        f = bf.objective(u, int(g.u0[gi]), g.c0[gi], g.c_su[gi], g.c_sd[gi], rho, ubar, y, z)
        assert f <= best + 1e-12 * abs(best)
        su, sd = bf.derived(u, int(g.u0[gi]))
        assert np.array_equal(post["u_su"][:, gi], su) and np.array_equal(post["u_sd"][:, gi], sd)


def test_adaptive_penalty_rule_and_state():
    """Residual balancing: after each check the three penalties are scaled by
    2 when r_p > 10 r_d, by 1/2 when r_d > 10 r_p, else kept; the penalties
    travel with the state (an oracle created with the scaled penalties, given
    the same state, sweeps identically)."""
    from paper_2310_13145_b300 import synth
    g = synth.config_instances("c1_9bus_T6")[0]
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, rho_every=1))
    changes = 0
    for _ in range(60):
        st0 = oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
        o.sweep()
        st1 = oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
        r = o.residuals()
        want = 2.0 if (r["r_p"] > 10 * r["r_d"] and st0["rho_log"] < 6) else (
            0.5 if (r["r_d"] > 10 * r["r_p"] and st0["rho_log"] > -6) else 1.0)
        if st1["done"]:
            want = 1.0
        assert abs(st1["rho_log"]) <= 6
        for name in ("rho_pq", "rho_va", "rho_uc"):
            assert st1[name] == st0[name] * want
        changes += want != 1.0
    assert changes > 0
    # the state's penalties drive the sweep
    st = o.state_vector()
    s = oracle.unpack_state(st, g.T, g.n_gen, g.n_branch, g.n_bus)
    o2 = oracle.Oracle(g, oracle.default_params(rho=(s["rho_pq"], s["rho_va"], s["rho_uc"]), rho_every=1))
    o2.set_state(st)
    o.sweep()
    o2.sweep()
    assert np.array_equal(o.state_vector(), o2.state_vector())


def test_converged_instance_takes_no_further_sweep():
    """Algorithm 1 ends at convergence: once a sweep has met both stopping
    tests (r_p, r_d <= eps_in and z_rms <= eps_out), further sweep calls
    leave the iterate and the residual record as they were."""
    g = synth.config_instances("c1_9bus_T6")[0]
    o = oracle.Oracle(g)
    for _ in range(60):
        o.sweep(50)
        if oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)["done"]:
            break
    st = oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
    assert st["done"] == 1.0
    r = o.residuals()
    assert r["r_p"] <= 1e-4 and r["r_d"] <= 1e-4 and r["z_rms"] <= 1e-4
    vec = o.state_vector()
    o.sweep(5)
    assert np.array_equal(o.state_vector(), vec)
    assert o.residuals() == r
