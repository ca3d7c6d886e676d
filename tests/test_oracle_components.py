"""Pins of the oracle's component solvers against independent methods.

- generator (R5): the nine-variable problem with the six slacks kept explicit
  (rows of Eq. pg_lo .. ramp_up as written) solved by scipy's bounded
  L-BFGS-B, and the KKT conditions of that problem at the oracle's point;
- duplicate-UC box QP (R7): scipy bounded least squares and a dense grid;
- bus projection (R8): a dense KKT solve of the equality-constrained QP;
- line subproblem (R6): an exact AC point must be returned exactly; at
  random targets the constrained KKT conditions (finite differences), h = 0,
  and a dense grid in polar coordinates around the solution (points that
  satisfy the product and angle equations exactly) must find nothing better.
"""
import numpy as np
import pytest
from scipy.optimize import lsq_linear, minimize

import oracle

# ------------------------------------------------------------------ generator


def gen_objective(x, prm, tg, has_prev):
    c2, c1, rho, pmax, qlo, qhi, p0 = prm
    p, q, ph, spl, spu, sql, squ, srd, sru = x
    if not has_prev:
        ph = p0
    t_pl, t_pu, t_ql, t_qu, t_rd, t_ru, t_gp, t_gq, t_tc = tg
    r = [p - spl - t_pl, p + spu - t_pu, q - sql - t_ql, q + squ - t_qu, p - ph - srd - t_rd, p - ph + sru - t_ru,
         p - t_gp, q - t_gq]
    f = c2 * p * p + c1 * p + 0.5 * rho * sum(v * v for v in r)
    if has_prev:
        f += 0.5 * rho * (ph - t_tc) ** 2
    return f


def gen_grad(x, prm, tg, has_prev):
    c2, c1, rho, pmax, qlo, qhi, p0 = prm
    p, q, ph, spl, spu, sql, squ, srd, sru = x
    if not has_prev:
        ph = p0
    t_pl, t_pu, t_ql, t_qu, t_rd, t_ru, t_gp, t_gq, t_tc = tg
    e = np.array([p - spl - t_pl, p + spu - t_pu, q - sql - t_ql, q + squ - t_qu, p - ph - srd - t_rd,
                  p - ph + sru - t_ru, p - t_gp, q - t_gq])
    g = np.zeros(9)
    g[0] = 2 * c2 * p + c1 + rho * (e[0] + e[1] + e[4] + e[5] + e[6])
    g[1] = rho * (e[2] + e[3] + e[7])
    g[2] = (rho * (-e[4] - e[5] + (ph - t_tc))) if has_prev else 0.0
    g[3], g[4], g[5], g[6], g[7], g[8] = -rho * e[0], rho * e[1], -rho * e[2], rho * e[3], -rho * e[4], rho * e[5]
    return g


def _gen_case(rng, has_prev):
    rho = float(rng.choice([5e3, 5e4]))
    pmax = rng.uniform(0.5, 4)
    Qmin, Qmax = -0.3 * pmax, 0.5 * pmax
    prm = [rng.uniform(50, 500), rng.uniform(1000, 4000), rho, pmax, min(0.0, Qmin), Qmax, 0.5 * pmax]
    # targets spread so that every row regime occurs
    tg = [rng.uniform(-0.2, 1.2) * pmax for _ in range(2)] + [rng.uniform(-0.5, 0.6) * pmax for _ in range(2)] + \
         [rng.uniform(-0.8, 0.8) * pmax for _ in range(2)] + [rng.uniform(-0.2, 1.2) * pmax,
                                                               rng.uniform(-0.4, 0.6) * pmax,
                                                               rng.uniform(-0.2, 1.2) * pmax]
    return prm, tg


def _bounds(prm, has_prev):
    c2, c1, rho, pmax, qlo, qhi, p0 = prm
    return [(0, pmax), (qlo, qhi), (0, pmax) if has_prev else (p0, p0)] + [(0, None)] * 6


@pytest.mark.parametrize("seed", range(30))
def test_gen_kkt_and_independent_minimiser(seed):
    rng = np.random.default_rng(seed)
    has_prev = bool(seed % 3)
    prm, tg = _gen_case(rng, has_prev)
    out = oracle.gen_solve(prm, has_prev, tg)
    x = out.copy()
    if not has_prev:
        x[2] = prm[6]
    # KKT of the 9-variable bound-constrained convex QP (projected gradient)
    g = gen_grad(x, prm, tg, has_prev)
    bnds = _bounds(prm, has_prev)
    scale = prm[2] * max(1.0, np.abs(tg).max())
    for i, (lo, hi) in enumerate(bnds):
        lo = -np.inf if lo is None else lo
        hi = np.inf if hi is None else hi
        pg = np.clip(x[i] - g[i] / scale, lo, hi) - x[i]
        assert abs(pg) <= 1e-12 * max(1.0, abs(x[i])) + 1e-13, (i, pg, x, g)
    # independent minimiser
    x0 = np.array([0.5 * prm[3], 0.0, 0.5 * prm[3] if has_prev else prm[6]] + [0.0] * 6)
    res = minimize(gen_objective, x0, args=(prm, tg, has_prev), jac=gen_grad, method="L-BFGS-B", bounds=bnds,
                   options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    f_or = gen_objective(x, prm, tg, has_prev)
    assert f_or <= res.fun + 1e-9 * max(1.0, abs(res.fun))
    assert np.allclose(x[:3], res.x[:3], rtol=0, atol=1e-5 * prm[3])


def test_gen_no_active_slack_is_closed_form():
    rho, pmax = 5e3, 3.0
    prm = [100.0, 2000.0, rho, pmax, -0.9, 1.5, 1.5]
    p_star = (rho * 1.2 - 2000.0) / (2 * 100.0 + rho)
    # slack rows far away: pl below, pu above, ramp window wide
    tg = [-10.0, 10.0, -10.0, 10.0, -10.0, 10.0, 1.2, 0.3, 0.7]
    out = oracle.gen_solve(prm, True, tg)
    assert abs(out[0] - p_star) < 1e-14 and abs(out[2] - 0.7) < 1e-15 and abs(out[1] - 0.3) < 1e-15
    assert np.all(out[3:] > 0)  # every slack strictly positive: every row exactly satisfied


# ------------------------------------------------------------------ box QP


@pytest.mark.parametrize("seed", range(30))
def test_boxqp_matches_bounded_least_squares(seed):
    rng = np.random.default_rng(100 + seed)
    n = 2 + seed % 2
    A = rng.normal(0, 1, (n + 4, n)) * rng.uniform(0.1, 10, n + 4)[:, None]
    m = rng.normal(0.5, 1.0, n + 4)
    H = A.T @ A
    g = A.T @ m
    x = oracle.boxqp(H, g)
    ref = lsq_linear(A, m, bounds=(0, 1), method="bvls", tol=1e-15)
    f = lambda v: 0.5 * v @ H @ v - g @ v
    assert f(x) <= f(ref.x) + 1e-12 * max(1, abs(f(ref.x)))
    assert np.allclose(x, ref.x, atol=1e-9)
    gr = H @ x - g
    for i in range(n):
        if x[i] <= 0:
            assert gr[i] >= -1e-9 * np.abs(H).max()
        elif x[i] >= 1:
            assert gr[i] <= 1e-9 * np.abs(H).max()
        else:
            assert abs(gr[i]) <= 1e-9 * np.abs(H).max()


def test_boxqp_dense_grid_2d():
    rng = np.random.default_rng(5)
    A = rng.normal(0, 1, (5, 2))
    m = rng.normal(0.3, 1.0, 5)
    H, g = A.T @ A, A.T @ m
    x = oracle.boxqp(H, g)
    u = np.linspace(0, 1, 801)
    X, Y = np.meshgrid(u, u, indexing="ij")
    F = 0.5 * (H[0, 0] * X * X + 2 * H[0, 1] * X * Y + H[1, 1] * Y * Y) - g[0] * X - g[1] * Y
    assert 0.5 * x @ H @ x - g @ x <= F.min() + 1e-14


# ------------------------------------------------------------------ bus


@pytest.mark.parametrize("seed", range(20))
def test_bus_matches_dense_kkt(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 12))
    W = rng.uniform(1e3, 1e5, n)
    m = rng.normal(0, 1, n)
    aP = rng.choice([-1.0, 0.0, 1.0], n)
    aQ = np.where(aP == 0, rng.choice([-1.0, 1.0], n), 0.0)
    aP[0], aQ[0] = -rng.uniform(0, 0.1), rng.uniform(0, 0.1)  # shunt on w
    Pd, Qd = rng.normal(0, 1), rng.normal(0, 0.5)
    v = oracle.bus_solve(W, m, aP, aQ, Pd, Qd)
    K = np.zeros((n + 2, n + 2))
    K[:n, :n] = np.diag(W)
    K[:n, n], K[n, :n] = aP, aP
    K[:n, n + 1], K[n + 1, :n] = aQ, aQ
    rhs = np.concatenate([W * m, [Pd, Qd]])
    ref = np.linalg.solve(K, rhs)[:n]
    assert np.allclose(v, ref, rtol=1e-12, atol=1e-12)
    assert abs(aP @ v - Pd) < 1e-12 and abs(aQ @ v - Qd) < 1e-12


# ------------------------------------------------------------------ line


def _line(rng, r=None, x=None, rate=None, bc=0.0):
    r = rng.uniform(0.005, 0.05) if r is None else r
    x = rng.uniform(0.05, 0.3) if x is None else x
    rate = rng.uniform(1, 3) if rate is None else rate
    z2 = r * r + x * x
    gs, bs = r / z2, -x / z2
    # (Gii, Bii, Gij, Bij, Gjj, Bjj, Gji, Bji) of the pi model with total charging bc
    Y = [gs, bs + 0.5 * bc, -gs, -bs, gs, bs + 0.5 * bc, -gs, -bs]
    lo = [0.81, 0.81, -1.21, -1.21, -2 * np.pi, -2 * np.pi, 0, 0]
    hi = [1.21, 1.21, 1.21, 1.21, 2 * np.pi, 2 * np.pi, rate * rate, rate * rate]
    return np.array(Y + [rate * rate] + lo + hi), (gs, bs, rate)


def polar_flows(gs, bs, Vi, Vj, ti, tj, bc=0.0):
    """Line flows from polar voltages: complex power V conj(I) of the pi
    model with series admittance gs + j bs and half the charging bc at each
    end."""
    Ui, Uj = Vi * np.exp(1j * ti), Vj * np.exp(1j * tj)
    y = gs + 1j * bs
    Sij = Ui * np.conj((y + 0.5j * bc) * Ui - y * Uj)
    Sji = Uj * np.conj((y + 0.5j * bc) * Uj - y * Ui)
    return Sij.real, Sij.imag, Sji.real, Sji.imag


def consensus(v_polar, gs, bs, tg, rpq, rva, bc=0.0):
    Vi, Vj, ti, tj = v_polar
    fl = polar_flows(gs, bs, Vi, Vj, ti, tj, bc)
    a = list(fl) + [Vi * Vi, Vj * Vj, ti, tj]
    return sum((rpq if k < 4 else rva) * 0.5 * (a[k] - tg[k]) ** 2 for k in range(8))


@pytest.mark.parametrize("bc", [0.0, 0.25])
@pytest.mark.parametrize("seed", range(8))
def test_line_exact_ac_point_is_returned(seed, bc):
    rng = np.random.default_rng(300 + seed)
    cst, (gs, bs, rate) = _line(rng, rate=5.0, bc=bc)
    Vi, Vj = rng.uniform(0.95, 1.05, 2)
    ti, tj = rng.uniform(-0.1, 0.1, 2)
    fl = polar_flows(gs, bs, Vi, Vj, ti, tj, bc)
    tgt = np.array(list(fl) + [Vi * Vi, Vj * Vj, ti, tj])
    d = ti - tj
    truth = np.array([Vi * Vi, Vj * Vj, Vi * Vj * np.cos(d), Vi * Vj * np.sin(d), ti, tj,
                      25.0 - fl[0] ** 2 - fl[1] ** 2, 25.0 - fl[2] ** 2 - fl[3] ** 2])
    v0 = truth + rng.normal(0, 1e-3, 8)
    rpq, rva = 5e4, 1e5
    v, mu, c, a, info = oracle.branch_solve(cst, tgt, rpq, rva, v0, np.zeros(4), 1e4 * rva)
    assert info[2] == 0
    assert np.allclose(v, truth, rtol=0, atol=1e-9), v - truth
    assert np.allclose(a, tgt, atol=1e-9)


@pytest.mark.parametrize("bc", [0.0, 0.25])
@pytest.mark.parametrize("seed", range(10))
def test_line_kkt_second_order_and_polar_grid(seed, bc):
    rng = np.random.default_rng(400 + seed)
    cst, (gs, bs, rate) = _line(rng, bc=bc)
    rpq, rva = 5e3, 1e4
    Vi, Vj = rng.uniform(0.95, 1.05, 2)
    ti, tj = rng.uniform(-0.2, 0.2, 2)
    fl = np.array(polar_flows(gs, bs, Vi, Vj, ti, tj, bc))
    # inconsistent targets: perturbed flows, voltages and angles
    tgt = np.concatenate([fl * rng.uniform(0.8, 1.2, 4) + rng.normal(0, 0.05, 4),
                          [Vi * Vi + rng.normal(0, 0.02), Vj * Vj + rng.normal(0, 0.02), ti + rng.normal(0, 0.02),
                           tj + rng.normal(0, 0.02)]])
    d = ti - tj
    v0 = np.array([Vi * Vi, Vj * Vj, Vi * Vj * np.cos(d), Vi * Vj * np.sin(d), ti, tj, 0.5, 0.5])
    v, mu, c, a, info = oracle.branch_solve(cst, tgt, rpq, rva, v0, np.zeros(4), 1e4 * rva)
    assert info[2] == 0
    lo, hi = cst[9:17], cst[17:25]
    Y = cst[:8]

    def f_of(w):
        p = [Y[0] * w[0] + Y[2] * w[2] + Y[3] * w[3], -Y[1] * w[0] - Y[3] * w[2] + Y[2] * w[3],
             Y[4] * w[1] + Y[6] * w[2] - Y[7] * w[3], -Y[5] * w[1] - Y[7] * w[2] - Y[6] * w[3]]
        a8 = p + [w[0], w[1], w[4], w[5]]
        return sum((rpq if k < 4 else rva) * 0.5 * (a8[k] - tgt[k]) ** 2 for k in range(8)), p

    def h_of(w):
        _, p = f_of(w)
        return np.array([w[2] ** 2 + w[3] ** 2 - w[0] * w[1], w[4] - w[5] - np.arctan2(w[3], w[2]),
                         p[0] ** 2 + p[1] ** 2 + w[6] - cst[8], p[2] ** 2 + p[3] ** 2 + w[7] - cst[8]])

    assert np.abs(h_of(v)).max() <= 1e-11
    # Lagrangian gradient by central differences (independent of the oracle's derivatives)
    lag = lambda w: f_of(w)[0] + mu @ h_of(w)
    eps = 1e-6
    gL = np.array([(lag(v + eps * e) - lag(v - eps * e)) / (2 * eps) for e in np.eye(8)])
    scale = rpq * 10
    for i in range(8):
        at_lo, at_hi = v[i] <= lo[i] + 1e-12, v[i] >= hi[i] - 1e-12
        if at_lo:
            assert gL[i] >= -1e-5 * scale
        elif at_hi:
            assert gL[i] <= 1e-5 * scale
        else:
            assert abs(gL[i]) <= 1e-5 * scale, (i, gL)
    # second order: objective over the manifold h0 = h1 = 0, parametrised by
    # polar voltages, on a dense grid in a small box around the solution
    Vi_s, Vj_s = np.sqrt(v[0]), np.sqrt(v[1])
    th_i, th_j = v[4], v[5]
    base = consensus((Vi_s, Vj_s, th_i, th_j), gs, bs, tgt, rpq, rva, bc)
    f_or, _ = f_of(v)
    assert abs(base - f_or) <= 1e-9 * max(1, f_or)
    g7 = np.linspace(-1e-3, 1e-3, 7)
    best = np.inf
    for a1 in g7:
        for a2 in g7:
            for a3 in g7:
                for a4 in g7:
                    Vi2, Vj2 = Vi_s + a1, Vj_s + a2
                    if not (0.9 <= Vi2 <= 1.1 and 0.9 <= Vj2 <= 1.1):
                        continue
                    fl2 = polar_flows(gs, bs, Vi2, Vj2, th_i + a3, th_j + a4, bc)
                    if fl2[0] ** 2 + fl2[1] ** 2 > cst[8] or fl2[2] ** 2 + fl2[3] ** 2 > cst[8]:
                        continue
                    best = min(best, consensus((Vi2, Vj2, th_i + a3, th_j + a4), gs, bs, tgt, rpq, rva, bc))
    assert best >= f_or - 1e-9 * max(1.0, f_or)


def test_relaxed_uc_step_is_the_box_minimiser():
    """The oracle's relaxed UC step (first phase of the UC warm start) puts
    each duplicate row at the minimiser of c u + rho/2 (u - tau)^2 on [0, 1],
    checked against a dense grid."""
    from paper_2310_13145_b300 import synth
    g = synth.config_instances("c1_9bus_T6")[0]
    o = oracle.Oracle(g)
    o.sweep(15)
    st = oracle.unpack_state(o.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
    rel = oracle.Oracle(g, oracle.default_params(rho=g.rho, uc_relax=1))
    rel.set_state(st)
    rel.sweep()
    out = oracle.unpack_state(rel.state_vector(), g.T, g.n_gen, g.n_branch, g.n_bus)
    rho = g.rho[2]
    grid = np.linspace(0.0, 1.0, 20001)
    for row, cost in (("on", g.c0), ("su", g.c_su), ("sd", g.c_sd)):
        tau = (st["ub_" + row] - st["gz_" + row]) - st["gy_" + row] / rho
        u = out["u_" + row]
        for t in range(g.T):
            for k in range(g.n_gen):
                f = cost[k] * grid + 0.5 * rho * (grid - tau[t, k]) ** 2
                best = grid[np.argmin(f)]
                assert abs(u[t, k] - best) <= 1e-4 + 1e-12, (row, t, k, u[t, k], best)
                assert 0.0 <= u[t, k] <= 1.0
