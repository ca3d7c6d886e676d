"""Free-running Algorithm 1 on the oracle (9-bus, T = 6) to convergence; the
converged point is checked against the model of Sec. II directly:
  - AC power flow in polar form from the bus copies (V = sqrt(wbar), thetabar)
    against the line subproblems' flows (Eq. acopf, flow equations);
  - power balance at every bus and period (Eq. uc_acopf_p/q_balance);
  - line limits and the product / angle equations at the line iterates;
  - the UC schedule against Eq. set:UC as written;
  - generator bounds and ramping with the schedule (Eq. coupling).
Violations must be of the order of the final coupling residual."""
import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf
from paper_2310_13145_b300 import synth


@pytest.fixture(scope="module", params=[False, True], ids=["plain", "shunts"])
def converged(request):
    # the second grid has bus shunts (one with both G^s and B^s) and line
    # charging on most lines
    g = synth.config_instances("c1_9bus_T6", shunts=request.param)[0]
    o = oracle.Oracle(g)
    for k in range(6000):
        o.sweep()
        if o.state()["done"]:
            break
    return g, o, o.state(), o.residuals(), k + 1


def _polar(gs, bs, Vi, Vj, d, bc=0.0):
    # pi model: series admittance gs + j bs, half the charging bc at each end
    pij = gs * Vi * Vi - Vi * Vj * (gs * np.cos(d) + bs * np.sin(d))
    qij = -(bs + 0.5 * bc) * Vi * Vi - Vi * Vj * (gs * np.sin(d) - bs * np.cos(d))
    pji = gs * Vj * Vj - Vi * Vj * (gs * np.cos(d) - bs * np.sin(d))
    qji = -(bs + 0.5 * bc) * Vj * Vj + Vi * Vj * (gs * np.sin(d) + bs * np.cos(d))
    return np.stack([pij, qij, pji, qji])


def test_converges(converged):
    g, o, st, r, n = converged
    assert st["done"] == 1.0, r
    assert max(r["r_p"], r["r_d"], r["z_rms"]) <= 1e-4


def test_ac_power_flow_in_polar_form(converged):
    g, o, st, r, n = converged
    tol = 30 * r["inf_norm"]
    GA, GB, BA, BB = o.rows()
    V = np.sqrt(st["wbar"])
    for l in range(g.n_branch):
        i, j = g.br_from[l], g.br_to[l]
        z2 = g.br_r[l] ** 2 + g.br_x[l] ** 2
        fl = _polar(g.br_r[l] / z2, -g.br_x[l] / z2, V[:, i], V[:, j], st["thbar"][:, i] - st["thbar"][:, j],
                    g.br_b[l])
        assert np.abs(fl - BA[:4, :, l]).max() <= tol, l
        assert np.abs(fl - np.stack([st["fb%d" % k][:, l] for k in range(4)])).max() <= tol, l


def test_power_balance(converged):
    g, o, st, r, n = converged
    for t in range(g.T):
        for i in range(g.n_bus):
            gens = np.nonzero(g.gen_bus == i)[0]
            P = st["pbar"][t, gens].sum() - g.Pd[t, i] - g.Gs[i] * st["wbar"][t, i]
            Q = st["qbar"][t, gens].sum() - g.Qd[t, i] + g.Bs[i] * st["wbar"][t, i]
            for l in range(g.n_branch):
                if g.br_from[l] == i:
                    P -= st["fb0"][t, l]; Q -= st["fb1"][t, l]
                if g.br_to[l] == i:
                    P -= st["fb2"][t, l]; Q -= st["fb3"][t, l]
            assert abs(P) < 1e-11 and abs(Q) < 1e-11


def test_line_constraints(converged):
    g, o, st, r, n = converged
    v = [st["v%d" % k] for k in range(8)]
    assert np.abs(v[2] ** 2 + v[3] ** 2 - v[0] * v[1]).max() < 1e-10
    assert np.abs(v[4] - v[5] - np.arctan2(v[3], v[2])).max() < 1e-10
    GA, GB, BA, BB = o.rows()
    rate2 = g.br_rate ** 2
    assert (BA[0] ** 2 + BA[1] ** 2 <= rate2 + 1e-9).all() and (BA[2] ** 2 + BA[3] ** 2 <= rate2 + 1e-9).all()
    assert (v[0] >= g.Vmin[g.br_from] ** 2 - 1e-12).all() and (v[0] <= g.Vmax[g.br_from] ** 2 + 1e-12).all()


def test_uc_schedule_and_coupling(converged):
    g, o, st, r, n = converged
    tol = 30 * r["inf_norm"]
    u, su, sd, p, q = st["u_on"], st["u_su"], st["u_sd"], st["p"], st["q"]
    for gi in range(g.n_gen):
        assert bf.feasible(u[:, gi].astype(int), int(g.u0[gi]), int(g.L0[gi]), int(g.F0[gi]), int(g.TU[gi]),
                           int(g.TD[gi]))
    assert (p >= g.Pmin * u - tol).all() and (p <= g.Pmax * u + tol).all()
    assert (q >= g.Qmin * u - tol).all() and (q <= g.Qmax * u + tol).all()
    pprev = np.vstack([g.p0[None, :], p[:-1]])
    uprev = np.vstack([g.u0[None, :], u[:-1]])
    assert (p - pprev <= g.RU * uprev + g.SU * su + tol).all()
    assert (p - pprev >= -g.RD * u - g.SD * sd - tol).all()
    # duplicates agree with the schedule
    assert np.abs(st["ub_on"] - u).max() <= tol
