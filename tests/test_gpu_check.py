"""The index-checked build (UCAC_CHECK=1, libucac_check.so).

Every index the sweep kernels take from a table (line-end slots, bus and
generator orders, work lists, instance lookups, granule ranges) is tested
against its buffer's extent before use.  These tests run the same sweeps on
the checked and the default library: no check may fail, and the iterates
must agree bit for bit (the checks change no arithmetic).  The failure path
-- a recorded site turned into an error by ucac_iterate -- is exercised with
ucac_check_inject, which records a site from a device thread without
touching any table.
"""
import numpy as np
import pytest

from paper_2310_13145_b300 import build, synth, warmstart

pytestmark = pytest.mark.gpu


def _with_lib(ucac, path, fn):
    old_path, old_lib = ucac.LIB_PATH, ucac._lib
    ucac.LIB_PATH, ucac._lib = path, None
    try:
        return fn()
    finally:
        ucac.LIB_PATH, ucac._lib = old_path, old_lib


def _run(ucac, grids, sweeps, params=None, warm=False):
    h = ucac.Handle(grids, params=params)
    if warm:
        h.set_warm_start(warmstart.init_params(5))
    rc = ucac.ucac_iterate(h.h, sweeps)
    states = [h.export(k) for k in range(len(grids))]
    h.close()
    return rc, states


def _cases(ucac):
    ragged = [synth.make_grid(n, nl, max(1, n // 3), T, seed=50 + n, rho=synth.RHO_TABLE["case300"])
              for n, nl, T in ((2, 1, 1), (5, 5, 3), (13, 16, 7), (31, 45, 5))]
    c2 = synth.config_instances("c2_118bus_T24x3")
    return [
        ("9-bus polar", synth.config_instances("c1_9bus_T6"), 12, None, False),
        ("9-bus W-form", synth.config_instances("c1_9bus_T6"), 12,
         ucac.ucac_default_params(line_form=ucac.UCAC_LINE_W), False),
        ("ragged batch", ragged, 8, None, False),
        ("118-bus batch, adaptive penalty", c2, 12, ucac.ucac_default_params(rho_every=3), False),
        ("118-bus batch, learned start", c2, 6, None, True),
    ]


def test_checked_build_runs_the_same_sweeps(ucac_mod):
    so_check = build.build(check=True)
    for name, grids, sweeps, params, warm in _cases(ucac_mod):
        rc_d, st_d = _run(ucac_mod, grids, sweeps, params, warm)
        rc_c, st_c = _with_lib(ucac_mod, so_check, lambda: _run(ucac_mod, grids, sweeps, params, warm))
        assert rc_c == rc_d and rc_c in (0, 1), (name, rc_c, rc_d)
        for k, (a, b) in enumerate(zip(st_d, st_c)):
            assert np.array_equal(a, b), (name, k)


def test_checked_build_reports_a_failed_check(ucac_mod):
    so_check = build.build(check=True)
    g = synth.config_instances("c1_9bus_T6")[0]

    def checked():
        h = ucac_mod.Handle([g])
        assert ucac_mod.ucac_iterate(h.h, 2) in (0, 1)
        assert ucac_mod.lib().ucac_check_inject(h.h, 77) == 0
        rc = ucac_mod.lib().ucac_iterate(h.h, 1)
        msg = ucac_mod.lib().ucac_last_error(h.h).decode()
        rc2 = ucac_mod.lib().ucac_iterate(h.h, 1)  # the record stays
        h.close()
        return rc, msg, rc2

    rc, msg, rc2 = _with_lib(ucac_mod, so_check, checked)
    assert rc == ucac_mod.UCAC_E_CUDA and "site 77" in msg and rc2 == ucac_mod.UCAC_E_CUDA
    # the default build has no checks to report
    h = ucac_mod.Handle([g])
    assert ucac_mod.lib().ucac_check_inject(h.h, 77) == ucac_mod.UCAC_E_ARG
    assert ucac_mod.ucac_iterate(h.h, 1) in (0, 1)
    h.close()
