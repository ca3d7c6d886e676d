"""Failure detection through the C ABI: the library's error statuses
(UCAC_E_NEWTON_MAXIT, UCAC_E_DIVERGED, UCAC_E_NAN) are produced, reported
per instance, stop only the instance concerned, and are returned by
ucac_iterate.  Every failure here is made on the host side of the API (an
iteration cap of 1, a divergence bound below the residual, a NaN written
into an imported state); no kernel is made to fault or hang."""
import numpy as np
import pytest

import oracle
from paper_2310_13145_b300 import synth

pytestmark = pytest.mark.gpu

E_NEWTON_MAXIT, E_NAN, E_DIVERGED = -4, -5, -6


def _g9():
    return synth.config_instances("c1_9bus_T6")[0]


# K_N = 1 caps the Newton loop of every multiplier round of both line forms.
# K_AL = 1 caps the W-form's multiplier rounds (its product and angle
# equations take several); the polar form's only multiplier equations are
# the line limits, which a free slack meets exactly, so on a lightly loaded
# grid its solves end in one round and K_AL = 1 caps nothing there.
CASES = [("polar", dict(K_N=1)), ("w", dict(K_N=1)), ("w", dict(K_AL=1))]


@pytest.mark.parametrize("form,cap", CASES, ids=["polar-K_N=1", "w-K_N=1", "w-K_AL=1"])
def test_iteration_cap_is_counted_then_reported(ucac_mod, form, cap):
    lf = ucac_mod.UCAC_LINE_POLAR if form == "polar" else ucac_mod.UCAC_LINE_W
    # counted only (default): sweeps go on with status 0 and the capped
    # solves are counted
    h = ucac_mod.Handle([_g9()], params=ucac_mod.ucac_default_params(line_form=lf, **cap))
    counts = []
    for _ in range(8):
        h.enqueue(1)
        r = h.residuals(0)
        assert r["status"] == 0, r
        counts.append(r["n_newton_maxit"])
    h.close()
    first = next(i for i, c in enumerate(counts) if c > 0)  # (StopIteration: nothing capped)
    # with stop_on_cap the instance stops with UCAC_E_NEWTON_MAXIT at the
    # first sweep that capped a solve, and takes no further sweep
    p = ucac_mod.ucac_default_params(line_form=lf, stop_on_cap=1, **cap)
    h = ucac_mod.Handle([_g9()], params=p)
    h.enqueue(first + 1)
    r = h.residuals(0)
    assert r["status"] == E_NEWTON_MAXIT and r["sweeps"] == first + 1 and r["n_newton_maxit"] == counts[first], r
    s = h.export(0)
    h.enqueue(3)
    assert np.array_equal(h.export(0), s) and h.residuals(0) == r
    st = oracle.unpack_state(s, 6, 3, 9, 9)
    assert st["done"] == 2.0
    with pytest.raises(ucac_mod.UcacError, match="error -4.*instance 0"):
        h.iterate(5)
    h.close()


def test_divergence_bound_stops_one_instance_of_a_batch(ucac_mod):
    # a bound between the two instances' first-sweep residuals: the first
    # instance stops with UCAC_E_DIVERGED, the second goes on
    grids = [_g9(), synth.config_instances("c2_118bus_T24x3", 1)[0]]
    h = ucac_mod.Handle(grids)
    h.enqueue(1)
    r0, r1 = h.residuals(0), h.residuals(1)
    h.close()
    lo, hi = sorted((max(r0["r_p"], r0["r_d"]), max(r1["r_p"], r1["r_d"])))
    assert hi > 1.5 * lo
    bound = np.sqrt(lo * hi)
    bad = 0 if max(r0["r_p"], r0["r_d"]) > bound else 1
    h = ucac_mod.Handle(grids, params=ucac_mod.ucac_default_params(div_bound=bound))
    h.enqueue(1)
    assert h.residuals(bad)["status"] == E_DIVERGED and h.residuals(1 - bad)["status"] == 0
    s_bad, s_ok = h.export(bad), h.export(1 - bad)
    h.enqueue(2)
    assert np.array_equal(h.export(bad), s_bad) and not np.array_equal(h.export(1 - bad), s_ok)
    assert h.residuals(1 - bad)["sweeps"] == 3 and h.residuals(bad)["sweeps"] == 1
    with pytest.raises(ucac_mod.UcacError, match=f"error -6.*instance {bad}"):
        h.iterate(1)
    h.close()


def test_nan_in_a_multiplier_gives_the_nan_status(ucac_mod):
    g = _g9()
    h = ucac_mod.Handle([g])
    h.enqueue(3)
    st = oracle.unpack_state(h.export(0), g.T, g.n_gen, g.n_branch, g.n_bus)
    st["by_pij"] = st["by_pij"].copy()
    st["by_pij"][2, 4] = np.nan
    h.import_(0, oracle.pack_state(st, g.T, g.n_gen, g.n_branch, g.n_bus))
    h.enqueue(1)
    r = h.residuals(0)
    assert r["status"] == E_NAN, r
    with pytest.raises(ucac_mod.UcacError, match="error -5"):
        h.iterate(2)
    h.close()


@pytest.mark.parametrize("form", ["polar", "w"])
def test_nan_line_slack_starts_at_zero(ucac_mod, form):
    # a NaN line-limit slack in an imported state: the line solve starts it
    # at 0 (the projection onto sigma >= 0), so the sweep stays finite and
    # matches the sweep from the same state with that slack set to 0
    lf = ucac_mod.UCAC_LINE_POLAR if form == "polar" else ucac_mod.UCAC_LINE_W
    g = _g9()
    p = ucac_mod.ucac_default_params(line_form=lf)
    h = ucac_mod.Handle([g], params=p)
    h.enqueue(3)
    st = oracle.unpack_state(h.export(0), g.T, g.n_gen, g.n_branch, g.n_bus)
    for k in ("v6", "v7"):
        st[k] = st[k].copy()
    st["v6"][1, 3] = np.nan
    st["v7"][4, 0] = -np.nan
    bad = oracle.pack_state(st, g.T, g.n_gen, g.n_branch, g.n_bus)
    st["v6"][1, 3] = 0.0
    st["v7"][4, 0] = 0.0
    zero = oracle.pack_state(st, g.T, g.n_gen, g.n_branch, g.n_bus)
    h.import_(0, bad)
    h.enqueue(1)
    a, ra = h.export(0), h.residuals(0)
    h.import_(0, zero)
    h.enqueue(1)
    b = h.export(0)
    h.close()
    assert ra["status"] == 0 and np.all(np.isfinite(a))
    assert np.array_equal(a, b)
