"""Pins of the oracle's outer update (Eq. step:outer, Sec. III-A) and of its
cold start (Sec. IV-A, Experiment Setting), rebuilt here from the paper's
statements rather than from the oracle's code.

Outer update (two-level ADMM, Sec. III-A): when the inner level terminates
at outer iteration k with slack z^k,
    lambda^{k+1} = Proj_[-lambda_max, lambda_max](lambda^k + beta^k z^k)
    beta^{k+1}   = tau beta^k   if |z^k| > theta |z^{k-1}|,   else beta^k,
where no |z^{k-1}| exists at the first outer iteration (so beta stays).
The library applies the step when the next sweep starts (the iterate it is
applied to is the one the inner level ended with).  The tests follow lambda
and beta through a run with a short inner cap, element by element and bit
for bit, and construct states on both sides of the strict comparison.

Cold start (Sec. IV-A): generator outputs and voltage magnitudes at the
middle of their bounds, voltage angles zero, line flows from those
voltages; x-bar = x and zero multipliers.  The flows are rebuilt here with
complex phasors and the pi-model admittance of each line.
"""
import numpy as np
import pytest

import oracle
from paper_2310_13145_b300 import synth

LAM = [f"glam_{r}" for r in oracle.GEN_ROWS] + [f"blam_{r}" for r in oracle.BR_ROWS]
ZS = [f"gz_{r}" for r in oracle.GEN_ROWS] + [f"bz_{r}" for r in oracle.BR_ROWS]
Z_OF = dict(zip(LAM, ZS))  # the slack z of each lambda's row


def _znorm(st):
    # |z|_2 over every coupling row (the temporal-copy row has no t = 0
    # instance; its entry stays zero and adds nothing)
    return float(np.sqrt(sum(float((np.asarray(st[k]) ** 2).sum()) for k in ZS)))


def _run(g, n, **kw):
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, **kw))
    sts = [o.state()]
    for _ in range(n):
        o.sweep()
        sts.append(o.state())
    return o, sts


@pytest.mark.parametrize("lam_max", [1e12, 2000.0])
def test_outer_update_rebuilt_by_hand(lam_max):
    g = synth.config_instances("c1_9bus_T6")[0]
    tau, theta, beta0 = 6.0, 0.8, 1e3
    _, sts = _run(g, 60, L_max=4, lam_max=lam_max, tau=tau, theta=theta, beta0=beta0)
    beta, beta_next, zprev = beta0, beta0, None
    lam = {k: np.zeros_like(np.asarray(sts[0][k])) for k in LAM}
    pending = None  # z^k of an inner level that ended in the previous sweep
    n_up = n_keep = n_clip = 0
    for n in range(1, len(sts)):
        s, prev = sts[n], sts[n - 1]
        if pending is not None:
            # step applied when the next sweep starts, with beta^k (not beta^{k+1})
            for k in LAM:
                v = lam[k] + beta * pending[Z_OF[k]]
                n_clip += int((np.abs(v) > lam_max).sum())
                lam[k] = np.clip(v, -lam_max, lam_max)
            beta = beta_next
            pending = None
        for k in LAM:
            assert np.array_equal(np.asarray(s[k]), lam[k]), (n, k)
        assert s["beta"] == beta, (n, s["beta"], beta)
        if s["k_outer"] > prev["k_outer"]:
            # the inner level terminated in sweep n: z^k is this sweep's z
            zk = _znorm(s)
            assert abs(s["zprev"] - zk) <= 1e-14 * zk, (n, s["zprev"], zk)
            if zprev is None:
                beta_next = beta  # first outer iteration: no |z^{k-1}|
            else:
                assert abs(zk - theta * zprev) > 1e-9 * zk  # decision away from the tie
                beta_next = tau * beta if zk > theta * zprev else beta
                n_up += beta_next != beta
                n_keep += beta_next == beta
            assert s["beta_next"] == beta_next, (n, s["beta_next"], beta_next)
            zprev = s["zprev"]
            pending = {k: np.asarray(s[k]).copy() for k in ZS}
            assert s["pending"] == 1.0
        else:
            assert s["pending"] == 0.0
    assert n_up >= 2 and n_keep >= 2  # both branches of the beta rule were taken
    if lam_max < 1e6:
        assert n_clip > 0  # the projection was active


def test_first_outer_iteration_keeps_beta():
    # a huge slack at the first termination must not raise beta: there is no
    # |z^{k-1}| to compare with
    g = synth.config_instances("c1_9bus_T6")[0]
    o, sts = _run(g, 4, L_max=4)
    s = sts[4]
    assert s["k_outer"] == 1.0 and s["zprev"] > 1.0
    assert s["beta_next"] == s["beta"] == 1e3


def _state_before_termination(g, theta):
    # a state two sweeps after an outer update, so that the next sweep
    # terminates the inner level again (L_max = 3) with a previous |z| known
    o = oracle.Oracle(g, oracle.default_params(rho=g.rho, L_max=3, theta=theta))
    o.sweep(3 + 2)
    st = o.state()
    assert st["k_outer"] == 1.0 and st["l_inner"] == 2.0 and st["zprev"] > 0.0
    return o, st


def test_beta_rule_comparison_is_strict():
    # theta = 1/2 makes theta * Z exact: Z = 2 |z^k| puts |z^k| exactly on
    # the threshold (no increase), the next double below puts it above
    g = synth.config_instances("c1_9bus_T6")[0]
    o, st = _state_before_termination(g, 0.5)
    beta = st["beta"]
    o.sweep()
    zk = o.state()["zprev"]
    assert o.state()["k_outer"] == 2.0
    for zp, expect in ((2.0 * zk, beta), (np.nextafter(2.0 * zk, 0.0), 6.0 * beta),
                       (np.nextafter(2.0 * zk, np.inf), beta)):
        s = dict(st)
        s["zprev"] = float(zp)
        o.set_state(s)
        o.sweep()
        r = o.state()
        assert r["zprev"] == zk  # same sweep, same |z^k|
        assert r["beta_next"] == expect, (zp, zk, r["beta_next"], expect)


def test_beta_rule_uses_the_norm_not_the_rms():
    # the rule compares 2-norms of z at consecutive terminations; an RMS (or
    # any rescaled) norm stored in place of |z^k| fails the first check
    g = synth.config_instances("c1_9bus_T6")[0]
    o, st = _state_before_termination(g, 0.8)
    o.sweep()
    s = o.state()
    assert abs(s["zprev"] - _znorm(s)) <= 1e-14 * _znorm(s)


# ---------------------------------------------------------------- cold start
def _cold_grid():
    # the 9-bus grid with per-bus voltage bands (so that |V| mid != 1), line
    # charging, bus shunts and one generator with a positive reactive floor
    # (so that the q interval [min(0, Qmin), Qmax] differs from [Qmin, Qmax])
    g = synth.config_instances("c1_9bus_T6")[0].copy()
    r = np.random.Generator(np.random.Philox(7))
    g.Vmin = r.uniform(0.90, 0.97, g.n_bus)
    g.Vmax = r.uniform(1.02, 1.10, g.n_bus)
    g.br_b = r.uniform(0.02, 0.3, g.n_branch)
    g.Gs = r.uniform(0.0, 0.05, g.n_bus)
    g.Bs = r.uniform(-0.1, 0.2, g.n_bus)
    g.Qmin = g.Qmin.copy()
    g.Qmin[1] = 0.1 * g.Pmax[1]
    return g


def _flows_phasor(g, V):
    """p_ij, q_ij, p_ji, q_ji of every line from complex bus voltages V
    (pi model: series y = 1/(r + jx), half the charging b at each end)."""
    y = 1.0 / (g.br_r + 1j * g.br_x)
    Vi, Vj = V[g.br_from], V[g.br_to]
    Iij = (y + 0.5j * g.br_b) * Vi - y * Vj
    Iji = (y + 0.5j * g.br_b) * Vj - y * Vi
    Sij, Sji = Vi * np.conj(Iij), Vj * np.conj(Iji)
    return Sij.real, Sij.imag, Sji.real, Sji.imag


def test_cold_start_rebuilt_from_the_text():
    g = _cold_grid()
    o = oracle.Oracle(g)
    s = o.state()
    T = g.T
    rmax = max(g.rho[0], g.rho[1])
    c0 = oracle.default_params().c_init_rel * rmax
    pmid = 0.5 * (0.0 + g.Pmax)                      # p in [0, Pmax]
    qmid = 0.5 * (np.minimum(0.0, g.Qmin) + g.Qmax)  # q in [min(0, Qmin), Qmax]
    Vmid = 0.5 * (g.Vmin + g.Vmax)
    close = lambda a, b: np.allclose(a, b, rtol=1e-15, atol=1e-15)
    assert close(s["p"], np.tile(pmid, (T, 1))) and close(s["pbar"], s["p"])
    assert close(s["q"], np.tile(qmid, (T, 1))) and close(s["qbar"], s["q"])
    # phat is the local copy of the previous period's output: p_0 at t = 1
    assert close(s["ph"][0], g.p0) and close(s["ph"][1:], np.tile(pmid, (T - 1, 1)))
    for f in ("s_pl", "s_pu", "s_ql", "s_qu", "s_rd", "s_ru", "u_su", "u_sd", "ub_su", "ub_sd"):
        assert not np.any(s[f]), f
    assert np.all(s["u_on"] == 1.0) and np.all(s["ub_on"] == 1.0)
    # W-form line variables at the flat start: w = |V|^2, wR = |V_i||V_j|,
    # wI = 0, angles 0
    i, j = g.br_from, g.br_to
    assert close(s["v0"], np.tile(Vmid[i] ** 2, (T, 1))) and close(s["v1"], np.tile(Vmid[j] ** 2, (T, 1)))
    assert close(s["v2"], np.tile(Vmid[i] * Vmid[j], (T, 1)))
    for f in ("v3", "v4", "v5"):
        assert not np.any(s[f]), f
    assert close(s["wbar"], np.tile(Vmid ** 2, (T, 1))) and not np.any(s["thbar"])
    # flows from the initial voltages (complex power of the pi model)
    F = _flows_phasor(g, Vmid.astype(complex))
    for k in range(4):
        assert np.allclose(s[f"fb{k}"], np.tile(F[k], (T, 1)), rtol=1e-13, atol=1e-14), k
    # line-limit slacks at their minimiser sigma = clip(rate^2 - |S|^2, 0, rate^2)
    r2 = g.br_rate ** 2
    for k, (a, b) in ((6, (F[0], F[1])), (7, (F[2], F[3]))):
        assert np.allclose(s[f"v{k}"], np.tile(np.clip(r2 - a * a - b * b, 0.0, r2), (T, 1)), rtol=1e-13,
                           atol=1e-14)
    # zero multipliers; the line penalty at its initial value
    for k in list(s):
        if k[:3] in ("gy_", "gz_", "by_", "bz_") or k[:4] in ("glam", "blam") or k.startswith("mu"):
            assert not np.any(s[k]), k
    assert np.all(s["cpen"] == c0)
    assert s["beta"] == s["beta_next"] == 1e3 and s["zprev"] == -1.0
    assert s["k_outer"] == s["l_inner"] == s["pending"] == s["done"] == 0.0


def test_cold_start_flows_satisfy_polar_power_flow():
    # the same flows in the polar form of the power-flow equations with all
    # angles zero: p_ij = G_ii V_i^2 + V_i V_j G_ij, q_ij = -B_ii V_i^2 - V_i V_j B_ij
    g = _cold_grid()
    s = oracle.Oracle(g).state()
    y = 1.0 / (g.br_r + 1j * g.br_x)
    Gii, Bii = y.real, y.imag + 0.5 * g.br_b
    Gij, Bij = -y.real, -y.imag
    V = 0.5 * (g.Vmin + g.Vmax)
    Vi, Vj = V[g.br_from], V[g.br_to]
    pij = Gii * Vi ** 2 + Vi * Vj * Gij
    qij = -Bii * Vi ** 2 - Vi * Vj * Bij
    pji = Gii * Vj ** 2 + Vi * Vj * Gij
    qji = -Bii * Vj ** 2 - Vi * Vj * Bij
    for k, ref in enumerate((pij, qij, pji, qji)):
        assert np.allclose(s[f"fb{k}"][0], ref, rtol=1e-13, atol=1e-14), k
