"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Lockstep: the oracle is given the library's exported iterate, runs one sweep,
and the two results are compared field by field (continuous fields within a
normwise relative 1e-9, UC decisions bit for bit).
"""
import numpy as np
import torch
import pytest

import oracle
from paper_2310_13145_b300 import synth
from tests._helpers import compare_states

pytestmark = pytest.mark.gpu


def _dims(g):
    return g.T, g.n_gen, g.n_branch, g.n_bus


# The polar line solver keeps no multipliers for the product and angle
# equations (they hold identically in its coordinates), so those two W-form
# multipliers and the W-form penalty are not compared for it; everything the
# ADMM iterates on is.  Its line-limit multipliers come from another path to
# the same KKT point and agree up to the inner stopping rule |h| <= eta.
POLAR_SKIP = ("mu0", "mu1", "cpen")


@pytest.fixture(params=["polar", "w"])
def line_form(request, ucac_mod):
    return ucac_mod.UCAC_LINE_POLAR if request.param == "polar" else ucac_mod.UCAC_LINE_W


def _lockstep(ucac, grids, sweeps, params=None, oparams=None, warm=0, check_instances=None, line_form=None,
              setup=None):
    if line_form is not None:
        params = params if params is not None else ucac.ucac_default_params()
        params.line_form = line_form
    polar = params is None or params.line_form == ucac.UCAC_LINE_POLAR
    skip = POLAR_SKIP if polar else ()
    mu_eta = (params.eta if params is not None else ucac.ucac_default_params().eta) if polar else None
    h = ucac.Handle(grids, params=params)
    if setup is not None:
        setup(h)
    if warm:
        h.enqueue(warm)
    orcs = {}
    ks = range(len(grids)) if check_instances is None else check_instances
    for k in ks:
        g = grids[k]
        op = oparams(g) if oparams else None
        orcs[k] = oracle.Oracle(g, op)
    worst = 0.0
    for s in range(sweeps):
        pre = {k: h.export(k) for k in ks}
        h.enqueue(1)
        for k in ks:
            o = orcs[k]
            o.set_state(pre[k])
            o.sweep()
            bad = compare_states(h.export(k), o.state_vector(), grids[k], skip=skip, mu_eta=mu_eta)
            assert not bad, f"sweep {s} instance {k}: {bad[:6]}"
    h.close()


def test_cold_start_matches(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    h = ucac_mod.Handle([g])
    o = oracle.Oracle(g)
    bad = compare_states(h.export(0), o.state_vector(), g, rtol=1e-14)
    assert not bad, bad
    h.close()


def test_cold_start_matches_ragged_batch(ucac_mod):
    # the device forms the cold start of every instance of a batch (uneven
    # sizes and horizons: the granule and slot indexing of each instance)
    grids = synth.config_instances("c4_batch64", 4)
    assert len({(g.n_bus, g.T) for g in grids}) > 1
    h = ucac_mod.Handle(grids)
    for k, g in enumerate(grids):
        bad = compare_states(h.export(k), oracle.Oracle(g).state_vector(), g, rtol=1e-14)
        assert not bad, (k, bad[:6])
    h.close()


def _coupled_buses(g):
    # buses whose P and Q balance multipliers are coupled in the x-bar
    # projection (Eq. step:opf_bar): the off-diagonal -G^s B^s / (deg rho_va)
    # of the 2x2 multiplier system is nonzero
    return np.flatnonzero((g.Gs != 0.0) & (g.Bs != 0.0))


def test_cold_start_matches_shunts(ucac_mod):
    # line charging enters the flows of the cold start (Eq. acopf, pi model)
    grids = synth.config_instances("c4_batch64", 4, shunts=True)
    assert all(np.any(g.br_b != 0.0) for g in grids)
    h = ucac_mod.Handle(grids)
    for k, g in enumerate(grids):
        bad = compare_states(h.export(k), oracle.Oracle(g).state_vector(), g, rtol=1e-14)
        assert not bad, (k, bad[:6])
    h.close()


def test_lockstep_9bus_shunts(ucac_mod, line_form):
    """Bus shunts and line charging (Eq. acopf, Sec. II-A): the bus
    kernel's coupled 2x2 multiplier solve and the charging terms of both
    line solvers, 40 sweeps in lockstep."""
    g = synth.config_instances("c1_9bus_T6", shunts=True)[0]
    assert _coupled_buses(g).size > 0 and np.count_nonzero(g.br_b) > 0
    _lockstep(ucac_mod, [g], 40, line_form=line_form)


def test_lockstep_9bus_shunts_with_outer_updates(ucac_mod, line_form):
    g = synth.config_instances("c1_9bus_T6", shunts=True)[0]
    p = ucac_mod.ucac_default_params(L_max=4)
    _lockstep(ucac_mod, [g], 20, params=p, oparams=lambda gg: oracle.default_params(rho=gg.rho, L_max=4), warm=60,
              line_form=line_form)


def test_lockstep_uneven_batch_shunts(ucac_mod, line_form):
    # four instances of the uneven batching workload with shunts and charging
    grids = synth.config_instances("c4_batch64", 4, shunts=True)
    assert all(_coupled_buses(g).size > 0 for g in grids)
    _lockstep(ucac_mod, grids, 3, warm=25, line_form=line_form)


def test_lockstep_9bus(ucac_mod, line_form):
    g = synth.config_instances("c1_9bus_T6")[0]
    _lockstep(ucac_mod, [g], 40, line_form=line_form)


def test_lockstep_9bus_late_with_outer_updates(ucac_mod, line_form):
    # small inner cap so that outer updates (lambda, beta) happen every few sweeps
    g = synth.config_instances("c1_9bus_T6")[0]
    p = ucac_mod.ucac_default_params(L_max=4)
    _lockstep(ucac_mod, [g], 25, params=p, oparams=lambda gg: oracle.default_params(rho=gg.rho, L_max=4), warm=60,
              line_form=line_form)


def test_lockstep_118bus_batch(ucac_mod, line_form):
    grids = synth.config_instances("c2_118bus_T24x3")
    _lockstep(ucac_mod, grids, 4, warm=10, line_form=line_form)


def test_lockstep_2000bus_late(ucac_mod):
    """One 2000-bus scenario 700 sweeps into a run to 1e-4, where line limits
    bind, penalties have grown to 1e8-1e10 and the polar solver's rarer
    paths run: variables fixed on a bound by the second Newton pass, solves
    finished from an extra evaluation, FP64-Hessian iterations, several AL
    rounds.  Two sweeps in lockstep with the oracle."""
    g = synth.config_instances("c5_2000bus_T24x16")[0]
    _lockstep(ucac_mod, [g], 2, warm=700, line_form=ucac_mod.UCAC_LINE_POLAR)
    # the regime is the late one: some solves take several AL rounds and the
    # Newton steps per solve are above the early runs' ~2
    h = ucac_mod.Handle([g])
    h.enqueue(701)
    r = h.residuals(0)
    solves = g.T * g.n_branch
    h.close()
    assert r["al"] > solves, (r["al"], solves)
    assert r["newton"] > 2.0 * solves, (r["newton"], solves)


def test_lockstep_uneven_batch(ucac_mod):
    # instances of the 64-instance batching workload (buses 93..416,
    # T in {12, 18, 24}) in one handle, 25 sweeps in, then 3 lockstep sweeps
    # of every instance against the oracle
    grids = synth.config_instances("c4_batch64", 4)
    assert len({g.T for g in grids}) > 1
    _lockstep(ucac_mod, grids, 3, warm=25)


def test_lockstep_ragged_small_instances(ucac_mod, line_form):
    # uneven batch: sizes that leave partial blocks in every kernel
    grids = [synth.make_grid(n, nl, max(1, n // 3), T, seed=50 + n, rho=synth.RHO_TABLE["case300"])
             for n, nl, T in ((2, 1, 1), (5, 5, 3), (13, 16, 7), (31, 45, 5))]
    _lockstep(ucac_mod, grids, 6, warm=3, line_form=line_form)


def test_batch_equals_single(ucac_mod):
    grids = synth.config_instances("c2_118bus_T24x3")
    hb = ucac_mod.Handle(grids)
    hb.enqueue(7)
    for k, g in enumerate(grids):
        hs = ucac_mod.Handle([g])
        hs.enqueue(7)
        assert np.array_equal(hs.export(0), hb.export(k)), k
        hs.close()
    hb.close()


def test_export_import_resume_is_bit_identical(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    h = ucac_mod.Handle([g])
    h.enqueue(5)
    s5 = h.export(0)
    h.enqueue(6)
    s11 = h.export(0)
    h2 = ucac_mod.Handle([g])
    h2.import_(0, s5)
    h2.enqueue(6)
    assert np.array_equal(h2.export(0), s11)
    h.close()
    h2.close()


def test_residual_record_matches_oracle(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    h = ucac_mod.Handle([g])
    h.enqueue(20)
    pre = h.export(0)
    h.enqueue(1)
    r = h.residuals(0)
    o = oracle.Oracle(g)
    o.set_state(pre)
    o.sweep()
    ro = o.residuals()
    for a, b in (("r_p", "r_p"), ("r_d", "r_d"), ("z_norm", "z_norm"), ("z_rms", "z_rms"),
                 ("inf_norm_viol", "inf_norm"), ("objective", "objective")):
        assert abs(r[a] - ro[b]) <= 1e-9 * max(abs(ro[b]), 1e-30), (a, r[a], ro[b])
    assert r["n_newton_maxit"] == 0
    h.close()


def test_full_size_2000bus_one_instance_lockstep(ucac_mod, line_form):
    """Largest workload in the bench's launch configuration (16 scenarios in
    one batch); one scenario's full sweep is recomputed by the oracle."""
    grids = synth.config_instances("c5_2000bus_T24x16")
    p = ucac_mod.ucac_default_params()
    p.line_form = line_form
    h = ucac_mod.Handle(grids, params=p)
    h.enqueue(3)
    k = 5
    pre = h.export(k)
    h.enqueue(1)
    o = oracle.Oracle(grids[k])
    o.set_state(pre)
    o.sweep()
    polar = line_form == ucac_mod.UCAC_LINE_POLAR
    bad = compare_states(h.export(k), o.state_vector(), grids[k], skip=POLAR_SKIP if polar else (),
                         mu_eta=p.eta if polar else None)
    assert not bad, bad[:6]
    h.close()


@pytest.mark.parametrize("every", [1, 5])
def test_lockstep_9bus_adaptive_penalty(ucac_mod, every):
    """Residual-balancing penalties (every `every` sweeps), in lockstep with
    the oracle: the decisions, the penalties and the rewritten targets."""
    g = synth.config_instances("c1_9bus_T6")[0]
    p = ucac_mod.ucac_default_params(rho_every=every)
    _lockstep(ucac_mod, [g], 40, params=p, oparams=lambda gg: oracle.default_params(rho=gg.rho, rho_every=every))


def test_lockstep_118bus_adaptive_penalty(ucac_mod):
    grids = synth.config_instances("c2_118bus_T24x3")
    p = ucac_mod.ucac_default_params(rho_every=10)
    _lockstep(ucac_mod, grids, 12, params=p, oparams=lambda gg: oracle.default_params(rho=gg.rho, rho_every=10),
              warm=35)


def test_adaptive_penalty_resume_bitwise(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0].copy()
    g.rho = tuple(100.0 * r for r in g.rho)  # mismatched on purpose: the balancing must act
    p = ucac_mod.ucac_default_params(rho_every=3)
    a = ucac_mod.Handle([g], params=p)
    a.enqueue(31)
    snap = a.export(0)
    st = oracle.unpack_state(snap, g.T, g.n_gen, g.n_branch, g.n_bus)
    assert st["rho_pq"] != g.rho[0]  # the penalties did move
    a.enqueue(20)
    b = ucac_mod.Handle([g], params=p)
    b.import_(0, snap)
    b.enqueue(20)
    assert np.array_equal(a.export(0), b.export(0))
    a.close()
    b.close()


def test_solution_readback(ucac_mod):
    # ucac_solution of every instance of a ragged batch: generator p, q, u_on
    # and bus w, theta are the iterate's own values; the line flows, in
    # [t][l][p_ij, q_ij, p_ji, q_ji] order, are those of its line variables
    # (the oracle's flow formula applied to the exported W-form variables)
    grids = synth.config_instances("c4_batch64", 3)
    h = ucac_mod.Handle(grids)
    h.enqueue(12)
    for k, g in enumerate(grids):
        sol = ucac_mod.ucac_solution(h.h, k, g.T, g.n_gen, g.n_bus, g.n_branch)
        buf = h.export(k)
        st = oracle.unpack_state(buf, g.T, g.n_gen, g.n_branch, g.n_bus)
        assert np.array_equal(sol["p"], st["p"]) and np.array_equal(sol["q"], st["q"])
        assert np.array_equal(sol["u_on"], (st["u_on"] != 0).astype(np.uint8))
        assert np.array_equal(sol["w"], st["wbar"]) and np.array_equal(sol["theta"], st["thbar"])
        o = oracle.Oracle(g)
        o.set_state(buf)
        _, _, BA, _ = o.rows()
        flows = np.moveaxis(BA[:4], 0, -1)  # [T][nl][4]
        assert sol["pf"].shape == flows.shape
        err = np.abs(sol["pf"] - flows).max()
        assert err <= 1e-9 * max(1.0, np.abs(flows).max()), (k, err)
        # the same bits into caller arrays (page-locked ones, as the bench's
        # end-to-end leg passes), and a wrong shape is refused
        pin = lambda shape, dt: torch.empty(shape, dtype=torch.from_numpy(np.zeros(0, dt)).dtype).pin_memory().numpy()  # noqa: E731
        out = ucac_mod.solution_arrays(g.T, g.n_gen, g.n_bus, g.n_branch, alloc=pin)
        sol2 = ucac_mod.ucac_solution(h.h, k, g.T, g.n_gen, g.n_bus, g.n_branch, out=out)
        assert sol2 is out and all(np.array_equal(sol[n], out[n]) for n in sol)
    bad = ucac_mod.solution_arrays(grids[0].T, grids[0].n_gen + 1, grids[0].n_bus, grids[0].n_branch)
    with pytest.raises(ucac_mod.UcacError):
        ucac_mod.ucac_solution(h.h, 0, grids[0].T, grids[0].n_gen, grids[0].n_bus, grids[0].n_branch, out=bad)
    h.close()


def test_converged_instance_is_frozen_in_a_batch(ucac_mod):
    # an instance that converges stops (Algorithm 1) while the rest of the
    # batch goes on; the oracle agrees that a converged state takes no sweep
    small = synth.config_instances("c1_9bus_T6")[0]
    big = synth.config_instances("c2_118bus_T24x3", 1)[0]
    h = ucac_mod.Handle([small, big])
    for _ in range(80):
        h.enqueue(25)
        if h.residuals(0)["status"] == 1:
            break
    r0 = h.residuals(0)
    assert r0["status"] == 1 and h.residuals(1)["status"] == 0
    s0, s1 = h.export(0), h.export(1)
    h.enqueue(10)
    assert np.array_equal(h.export(0), s0)
    assert h.residuals(0) == r0
    assert not np.array_equal(h.export(1), s1)
    o = oracle.Oracle(small)
    o.set_state(s0)
    o.sweep(3)
    assert np.array_equal(o.state_vector(), s0)
    h.close()


def test_work_order_changes_no_result(ucac_mod):
    """The polar line kernel takes the line-periods that met a bound or held
    a slack in the previous sweep first (their marks and list are cleared by
    a state import).  300 sweeps into the 118-bus batch -- voltage bounds
    and line limits bind by then -- a run that keeps its marks and a run
    that restarts from the exported state without them reach the same bits
    30 sweeps later."""
    grids = synth.config_instances("c2_118bus_T24x3")
    a = ucac_mod.Handle(grids)
    a.enqueue(300)
    snaps = [a.export(k) for k in range(len(grids))]
    a.enqueue(30)
    b = ucac_mod.Handle(grids)
    for k, s in enumerate(snaps):
        b.import_(k, s)
    b.enqueue(30)
    for k in range(len(grids)):
        assert np.array_equal(a.export(k), b.export(k)), k
        assert a.residuals(k)["newton"] == b.residuals(k)["newton"]
    a.close()
    b.close()


def test_lockstep_generator_q_pieces(ucac_mod):
    """The generator kernel takes q from the piece of its piecewise linear
    optimality condition that the condition's signs at the two breakpoints
    (the q-bound rows' targets) pick.  Multipliers of the q-bound and
    q-consensus rows are drawn so that the targets fall in every order --
    crossed ones (the slope-3 piece) included -- and one sweep from that
    state is compared with the oracle's."""
    g = synth.config_instances("c2_118bus_T24x3")[0]
    dims = _dims(g)
    h = ucac_mod.Handle([g])
    h.enqueue(20)
    st = oracle.unpack_state(h.export(0), *dims)
    rng = np.random.default_rng(11)
    rho = st["rho_pq"]
    span = np.maximum(g.Qmax - g.Qmin, 0.1)[None, :]
    for row in ("ql", "qu", "gq"):
        st["gy_" + row] = st["gy_" + row] + rho * span * rng.uniform(-1.5, 1.5, st["gy_" + row].shape)
    # targets t = b - z - y/rho of the q-bound rows (their x-bar values are
    # Qmin u_on and Qmax u_on): some must cross
    t_ql = g.Qmin[None, :] * st["ub_on"] - st["gz_ql"] - st["gy_ql"] / rho
    t_qu = g.Qmax[None, :] * st["ub_on"] - st["gz_qu"] - st["gy_qu"] / rho
    assert np.count_nonzero(t_ql > t_qu) > 100
    h.import_(0, oracle.pack_state(st, *dims))
    pre = h.export(0)
    h.enqueue(1)
    o = oracle.Oracle(g)
    o.set_state(pre)
    o.sweep()
    bad = compare_states(h.export(0), o.state_vector(), g, skip=POLAR_SKIP,
                         mu_eta=ucac_mod.ucac_default_params().eta)
    assert not bad, bad[:6]
    h.close()


def test_lockstep_uc_box_faces(ucac_mod):
    """The duplicate-UC box QPs solve each face from the free block's
    inverse, formed once per generator and penalty (k_prep_ucbar).
    Multipliers of every row of the box QPs drawn at the scale of the
    penalties move their minimisers onto every kind of face -- interior,
    edges, corners, through the pivots and the full enumeration -- and one
    sweep from that state is compared with the oracle's."""
    g = synth.config_instances("c2_118bus_T24x3")[1]
    dims = _dims(g)
    h = ucac_mod.Handle([g])
    h.enqueue(20)
    st = oracle.unpack_state(h.export(0), *dims)
    rng = np.random.default_rng(12)
    for row, rho in (("on", st["rho_uc"]), ("su", st["rho_uc"]), ("sd", st["rho_uc"]), ("pl", st["rho_pq"]),
                     ("pu", st["rho_pq"]), ("rd", st["rho_pq"]), ("ru", st["rho_pq"])):
        st["gy_" + row] = st["gy_" + row] + rho * rng.uniform(-2.0, 2.0, st["gy_" + row].shape)
    h.import_(0, oracle.pack_state(st, *dims))
    pre = h.export(0)
    h.enqueue(1)
    o = oracle.Oracle(g)
    o.set_state(pre)
    o.sweep()
    out = oracle.unpack_state(h.export(0), *dims)
    # the minimisers spread over the box: interior and bound values both occur
    ub = np.concatenate([out["ub_on"].ravel(), out["ub_sd"].ravel()])
    assert np.count_nonzero((ub > 1e-9) & (ub < 1 - 1e-9)) > 50 and np.count_nonzero(ub <= 0.0) > 50
    bad = compare_states(h.export(0), o.state_vector(), g, skip=POLAR_SKIP,
                         mu_eta=ucac_mod.ucac_default_params().eta)
    assert not bad, bad[:6]
    h.close()


def test_lockstep_line_solves_pushed_to_bounds(ucac_mod):
    """The polar line kernel takes the common Newton step with FP32 limit
    gradients and hands every other case -- a variable near a bound, a
    held slack, a shifted system, a trust-region step -- to the full step.
    Multipliers of the flow and voltage rows drawn at half the penalty's
    scale push many solves onto line limits and voltage bounds, so both
    paths run in one sweep; the sweep is compared with the oracle's.  (At
    twice the penalty's scale the targets sit ~2 p.u. from any feasible
    flow; the nonconvex line subproblems then have several KKT points and
    the two solvers, on their different routes, stop at different ones.)"""
    g = synth.config_instances("c2_118bus_T24x3")[2]
    dims = _dims(g)
    h = ucac_mod.Handle([g])
    h.enqueue(20)
    st = oracle.unpack_state(h.export(0), *dims)
    rng = np.random.default_rng(13)
    for row, rho, sc in (("pij", st["rho_pq"], 0.5), ("qij", st["rho_pq"], 0.5), ("pji", st["rho_pq"], 0.5),
                         ("qji", st["rho_pq"], 0.5), ("wi", st["rho_va"], 0.05), ("wj", st["rho_va"], 0.05)):
        st["by_" + row] = st["by_" + row] + rho * sc * rng.uniform(-1.0, 1.0, st["by_" + row].shape)
    h.import_(0, oracle.pack_state(st, *dims))
    pre = h.export(0)
    h.enqueue(1)
    o = oracle.Oracle(g)
    o.set_state(pre)
    o.sweep()
    out = oracle.unpack_state(h.export(0), *dims)
    # line limits bind (positive limit multipliers) on a good share of solves
    assert np.count_nonzero(out["mu2"] > 0) + np.count_nonzero(out["mu3"] > 0) > 100
    bad = compare_states(h.export(0), o.state_vector(), g, skip=POLAR_SKIP,
                         mu_eta=ucac_mod.ucac_default_params().eta)
    assert not bad, bad[:6]
    h.close()


def test_line_counts_sum_to_the_record(ucac_mod, line_form):
    """The per-solve device counters behind the Newton-iteration histograms:
    for every instance of a batch and both line forms, the Newton iterations
    and multiplier rounds stored per line-period sum to the instance's
    record of the same sweep, and every solve ran at least one multiplier
    round."""
    grids = synth.config_instances("c2_118bus_T24x3")
    h = ucac_mod.Handle(grids, params=ucac_mod.ucac_default_params(line_form=line_form))
    for sweeps in (1, 14):
        h.enqueue(sweeps)
        for k, g in enumerate(grids):
            nw, na = h.line_counts(k)
            r = h.residuals(k)
            assert nw.shape == (g.T, g.n_branch)
            assert int(nw.sum()) == r["newton"] and int(na.sum()) == r["al"], (k, sweeps)
            assert na.min() >= 1
            hist = ucac_mod.count_histogram(nw)
            assert sum(hist) == g.T * g.n_branch
    h.close()


def test_handles_with_different_horizons(ucac_mod):
    # the sweep's UC dynamic program keeps its tables in shared memory sized
    # by the handle's horizon; a later handle with a shorter horizon must not
    # break the sweeps the first one has captured (the kernel's shared-memory
    # limit is shared by all handles), and the two interleave bit for bit
    long_g = synth.make_grid(20, 30, 6, 96, seed=11)
    short_g = synth.make_grid(9, 12, 3, 6, seed=12)
    ref = ucac_mod.Handle([long_g])
    ref.enqueue(6)
    want = ref.export(0)
    ref.close()
    a = ucac_mod.Handle([long_g])
    a.enqueue(3)
    b = ucac_mod.Handle([short_g])
    b.enqueue(4)
    a.enqueue(3)
    assert np.array_equal(a.export(0), want)
    assert a.residuals(0)["status"] >= 0 and b.residuals(0)["status"] >= 0
    a.close()
    b.close()
