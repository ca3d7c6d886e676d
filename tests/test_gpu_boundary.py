"""Every entry point of the library's C boundary -- create, create_batch,
iterate, residuals, solution, set_warmstart (BF16 blob), state_export,
state_import, destroy, last_error -- called directly through ctypes with
plain pointers and sizes, as a C caller would."""
import ctypes as C

import numpy as np
import pytest

from paper_2310_13145_b300 import synth, warmstart

pytestmark = pytest.mark.gpu

_dp = C.POINTER(C.c_double)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def _bf16(p32):
    """Round-to-nearest-even FP32 -> BF16 bit patterns."""
    u = np.ascontiguousarray(p32, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def test_boundary_entry_points_through_ctypes(ucac_mod):
    u = ucac_mod
    L = u.lib()
    g = synth.config_instances("c1_9bus_T6")[0]
    g2 = synth.make_grid(13, 16, 4, 5, seed=63, rho=synth.RHO_TABLE["case300"])
    keep = []
    s1, s2 = u._grid_struct(g, keep), u._grid_struct(g2, keep)
    # ucac_create (params NULL = defaults, stream NULL)
    h = C.c_void_p()
    assert L.ucac_create(C.byref(s1), g.T, u.ucac_rho(*g.rho), None, None, C.byref(h)) == 0 and h.value
    # ucac_create_batch of two uneven instances with their own penalties
    hb = C.c_void_p()
    arr = (C.POINTER(u.ucac_grid) * 2)(C.pointer(s1), C.pointer(s2))
    hz = np.array([g.T, g2.T], np.int32)
    rs = (u.ucac_rho * 2)(u.ucac_rho(*g.rho), u.ucac_rho(*g2.rho))
    assert L.ucac_create_batch(arr, _ptr(hz, C.POINTER(C.c_int32)), rs, 2, None, None, C.byref(hb)) == 0
    # ucac_iterate, ucac_residuals
    assert L.ucac_iterate(h, 10) in (0, 1)
    rep = u.ucac_report()
    assert L.ucac_residuals(h, 0, C.byref(rep)) == 0 and rep.sweeps == 10 and rep.status == 0
    assert np.isfinite(rep.r_p) and rep.r_p > 0
    # ucac_solution into caller buffers (any may be NULL)
    T, ng, nb, nl = g.T, g.n_gen, g.n_bus, g.n_branch
    p, q, w, th = np.zeros((T, ng)), np.zeros((T, ng)), np.zeros((T, nb)), np.zeros((T, nb))
    pf, uon = np.zeros((T, nl, 4)), np.zeros((T, ng), np.uint8)
    assert L.ucac_solution(h, 0, _ptr(p), _ptr(q), _ptr(w), _ptr(th), _ptr(pf), _ptr(uon, C.POINTER(C.c_uint8))) == 0
    assert np.all(w > 0.5) and np.all(uon <= 1) and np.all(np.isfinite(pf))
    assert L.ucac_solution(h, 0, None, None, None, None, None, None) == 0
    # ucac_line_counts: per line-period Newton iterations and multiplier
    # rounds of the last sweep, summing to the record's counts
    nw, na = np.zeros((T, nl), np.uint16), np.zeros((T, nl), np.uint16)
    u16 = C.POINTER(C.c_uint16)
    assert L.ucac_line_counts(h, 0, _ptr(nw, u16), _ptr(na, u16)) == 0
    assert int(nw.sum()) == rep.newton and int(na.sum()) == rep.al and na.min() >= 1
    assert L.ucac_line_counts(h, 0, None, None) == 0
    assert L.ucac_line_counts(h, 5, None, None) == u.UCAC_E_ARG
    # ucac_state_export / ucac_state_import: resume instance 0 of the batch
    # from the single handle's iterate
    n = L.ucac_state_size(h, 0)
    buf = np.empty(n)
    assert L.ucac_state_export(h, 0, _ptr(buf), n) == 0
    assert L.ucac_state_import(hb, 0, _ptr(buf), n) == 0
    assert L.ucac_iterate(h, 3) in (0, 1) and L.ucac_iterate(hb, 3) in (0, 1)
    a, b = np.empty(n), np.empty(n)
    L.ucac_state_export(h, 0, _ptr(a), n)
    L.ucac_state_export(hb, 0, _ptr(b), n)
    assert np.array_equal(a, b)
    # a wrong size is rejected with a reason
    assert L.ucac_state_export(h, 0, _ptr(buf), n - 1) == u.UCAC_E_ARG
    assert L.ucac_last_error(h)
    # ucac_set_warmstart: a BF16 blob of the network
    blob = _bf16(warmstart.init_params(3))
    assert L.ucac_set_warmstart(h, C.c_void_p(blob.ctypes.data), blob.nbytes) == 0
    assert L.ucac_iterate(h, 2) in (0, 1)
    assert L.ucac_set_warmstart(h, C.c_void_p(blob.ctypes.data), blob.nbytes - 2) == u.UCAC_E_ARG
    assert b"BF16" in L.ucac_last_error(h)
    assert L.ucac_set_warmstart(h, None, 0) == 0
    # ucac_destroy (NULL ignored); ucac_last_error(NULL) after a failed create
    L.ucac_destroy(h)
    L.ucac_destroy(hb)
    L.ucac_destroy(None)
    bad = C.c_void_p()
    assert L.ucac_create(C.byref(s1), g.T + 1, u.ucac_rho(*g.rho), None, None, C.byref(bad)) == u.UCAC_E_GRID
    assert bad.value is None and L.ucac_last_error(None)


def test_bf16_blob_equals_fp32_params_of_the_same_values(ucac_mod):
    # the BF16 entry point widens exactly: the same network given as FP32
    # values of those BF16 numbers takes the same starts, bit for bit
    u = ucac_mod
    blob = _bf16(warmstart.init_params(5) * 0.5)
    p32 = (blob.astype(np.uint32) << 16).view(np.float32)
    g = synth.config_instances("c1_9bus_T6")[0]
    out = []
    for mode in ("bf16", "fp32"):
        h = u.Handle([g])
        h.enqueue(5)
        if mode == "bf16":
            u.ucac_set_warmstart(h.h, blob)
        else:
            h.set_warm_start(p32)
        h.enqueue(6)
        out.append((h.export(0), h.warm_start_stats(0)))
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
