"""Thin ctypes binding of the ucac C ABI (include/ucac.h), same names.

Argument marshalling only: every step of a sweep runs in the library's CUDA
kernels.  Loading fails loudly when libucac.so is missing; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libucac.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)

UCAC_OK, UCAC_CONVERGED = 0, 1
UCAC_E_ARG, UCAC_E_GRID, UCAC_E_CUDA, UCAC_E_NEWTON_MAXIT, UCAC_E_NAN, UCAC_E_DIVERGED = -1, -2, -3, -4, -5, -6
UCAC_N_KERNELS = 7
UCAC_LINE_W, UCAC_LINE_POLAR = 0, 1

# symbols declared in include/ucac.h
EXPORTS = ["ucac_default_params", "ucac_create", "ucac_create_batch", "ucac_instances", "ucac_iterate",
           "ucac_enqueue_sweeps", "ucac_residuals", "ucac_solution", "ucac_state_size", "ucac_state_export",
           "ucac_state_import", "ucac_kernel_times", "ucac_kernel_name", "ucac_ucdp_workspace_bytes", "ucac_ucdp", "ucac_ucdp_noalloc",
           "ucac_probe_fp64", "ucac_probe_cossin", "ucac_probe_dw", "ucac_autotune", "ucac_uc_warm_start", "ucac_mlp_param_count", "ucac_mlp_workspace_bytes", "ucac_mlp_forward",
           "ucac_mlp_grad", "ucac_mlp_adam", "ucac_line_features", "ucac_line_samples", "ucac_set_warm_start", "ucac_set_warmstart",
           "ucac_warm_start_stats", "ucac_line_counts", "ucac_check_inject",
           "ucac_destroy", "ucac_last_error"]


class ucac_grid(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("n_gen", C.c_int32), ("T", C.c_int32),
                ("ref_bus", C.c_int32)] + \
        [(n, _dp) for n in ("Pd", "Qd", "Gs", "Bs", "Vmin", "Vmax")] + \
        [(n, _ip) for n in ("br_from", "br_to")] + \
        [(n, _dp) for n in ("br_r", "br_x", "br_b", "br_rate")] + \
        [("gen_bus", _ip)] + \
        [(n, _dp) for n in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0", "c_su", "c_sd", "RU", "RD", "SU", "SD")] + \
        [(n, _ip) for n in ("TU", "TD", "u0", "L0", "F0")] + \
        [("p0", _dp), ("base_mva", C.c_double)]


class ucac_rho(C.Structure):
    _fields_ = [("pq", C.c_double), ("va", C.c_double), ("uc", C.c_double)]


class ucac_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("eps_in", "eps_out", "tau", "theta", "beta0", "lambda_max", "eta",
                                          "omega_rel", "c_init_rel", "c_max_rel", "rho_mu", "rho_tau")] + \
        [(n, C.c_int32) for n in ("K_AL", "K_N", "L_max", "check_every", "line_form", "uc_relax", "rho_every",
                                  "stop_on_cap")] + \
        [("div_bound", C.c_double)]


class ucac_report(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("r_p", "r_d", "z_norm", "z_rms", "inf_norm_viol", "objective", "beta")] + \
        [(n, C.c_int64) for n in ("sweeps", "outer", "newton", "al")] + \
        [("status", C.c_int32), ("n_newton_maxit", C.c_int32)] + \
        [(n, C.c_int64) for n in ("newton_total", "al_total")]


class UcacError(RuntimeError):
    pass


def lib():
    """Loads libucac.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise UcacError(f"{LIB_PATH} not found: build it with paper_2310_13145_b300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.ucac_default_params.argtypes = [C.POINTER(ucac_params)]
        L.ucac_default_params.restype = None
        L.ucac_create.argtypes = [C.POINTER(ucac_grid), C.c_int32, ucac_rho, C.POINTER(ucac_params), vp,
                                  C.POINTER(vp)]
        L.ucac_create_batch.argtypes = [C.POINTER(C.POINTER(ucac_grid)), _ip, C.POINTER(ucac_rho), C.c_int32,
                                        C.POINTER(ucac_params), vp, C.POINTER(vp)]
        L.ucac_instances.argtypes = [vp]
        L.ucac_instances.restype = C.c_int32
        L.ucac_iterate.argtypes = [vp, C.c_int32]
        L.ucac_enqueue_sweeps.argtypes = [vp, C.c_int32]
        L.ucac_residuals.argtypes = [vp, C.c_int32, C.POINTER(ucac_report)]
        L.ucac_solution.argtypes = [vp, C.c_int32, _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_uint8)]
        L.ucac_line_counts.argtypes = [vp, C.c_int32, C.POINTER(C.c_uint16), C.POINTER(C.c_uint16)]
        L.ucac_check_inject.argtypes = [vp, C.c_int32]
        L.ucac_state_size.argtypes = [vp, C.c_int32]
        L.ucac_state_size.restype = C.c_size_t
        L.ucac_state_export.argtypes = [vp, C.c_int32, _dp, C.c_size_t]
        L.ucac_state_import.argtypes = [vp, C.c_int32, _dp, C.c_size_t]
        L.ucac_kernel_times.argtypes = [vp, C.c_int32, _dp]
        L.ucac_kernel_name.argtypes = [C.c_int32]
        L.ucac_kernel_name.restype = C.c_char_p
        L.ucac_ucdp_workspace_bytes.argtypes = [C.c_int32, C.c_int32]
        L.ucac_ucdp_workspace_bytes.restype = C.c_size_t
        L.ucac_ucdp.argtypes = [C.c_int32, C.c_int32, C.c_double] + [vp] * 12 + [vp, C.c_size_t, vp]
        L.ucac_ucdp_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_double] + [vp] * 12 + [vp]
        L.ucac_probe_fp64.argtypes = [C.c_int32, vp, _dp]
        L.ucac_probe_cossin.argtypes = [C.c_int32, _dp, _dp, _dp]
        L.ucac_probe_dw.argtypes = [C.c_int32, C.c_int32, _dp, _dp, _dp, _dp]
        L.ucac_autotune.argtypes = [vp, C.c_int32, C.c_char_p, _ip]
        L.ucac_uc_warm_start.argtypes = [vp, C.c_int32, C.c_double]
        L.ucac_mlp_param_count.argtypes = []
        L.ucac_mlp_param_count.restype = C.c_int32
        L.ucac_mlp_workspace_bytes.argtypes = [C.c_int64]
        L.ucac_mlp_workspace_bytes.restype = C.c_size_t
        L.ucac_mlp_forward.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_size_t, vp]
        L.ucac_mlp_grad.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
        L.ucac_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_float, vp]
        L.ucac_line_features.argtypes = [vp, C.c_int32, C.POINTER(C.c_float), _dp]
        L.ucac_line_samples.argtypes = [vp, C.POINTER(C.c_float), _dp, _dp]
        L.ucac_set_warm_start.argtypes = [vp, C.POINTER(C.c_float)]
        L.ucac_set_warmstart.argtypes = [vp, vp, C.c_size_t]
        L.ucac_warm_start_stats.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64), _ip]
        L.ucac_destroy.argtypes = [vp]
        L.ucac_destroy.restype = None
        L.ucac_last_error.argtypes = [vp]
        L.ucac_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc, h=None):
    if rc < 0:
        msg = lib().ucac_last_error(h)
        raise UcacError(f"ucac error {rc}: {msg.decode() if msg else ''}")
    return rc


def ucac_default_params(**kw) -> ucac_params:
    p = ucac_params()
    lib().ucac_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _grid_struct(g, keep):
    def dd(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_dp)

    def ii(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        keep.append(a)
        return a.ctypes.data_as(_ip)

    s = ucac_grid()
    s.n_bus, s.n_branch, s.n_gen, s.T, s.ref_bus = g.n_bus, g.n_branch, g.n_gen, g.T, g.ref_bus
    for n in ("Pd", "Qd", "Gs", "Bs", "Vmin", "Vmax", "br_r", "br_x", "br_b", "br_rate", "Pmin", "Pmax", "Qmin",
              "Qmax", "c2", "c1", "c0", "c_su", "c_sd", "RU", "RD", "SU", "SD", "p0"):
        setattr(s, n, dd(getattr(g, n)))
    for n in ("br_from", "br_to", "gen_bus", "TU", "TD", "u0", "L0", "F0"):
        setattr(s, n, ii(getattr(g, n)))
    s.base_mva = g.base_mva
    return s


def ucac_create_batch(grids, horizons=None, rhos=None, params=None, stream=0):
    """Returns an opaque handle (c_void_p) for a batch of synth.Grid-like instances."""
    keep = []
    n = len(grids)
    structs = [_grid_struct(g, keep) for g in grids]
    arr = (C.POINTER(ucac_grid) * n)(*[C.pointer(s) for s in structs])
    hz = np.ascontiguousarray([g.T if horizons is None else horizons[k] for k, g in enumerate(grids)], np.int32)
    rs = (ucac_rho * n)(*[ucac_rho(*(g.rho if rhos is None else rhos[k])) for k, g in enumerate(grids)])
    out = C.c_void_p()
    p = C.byref(params) if params is not None else None
    _check(lib().ucac_create_batch(arr, hz.ctypes.data_as(_ip), rs, n, p, C.c_void_p(stream), C.byref(out)))
    return out


def ucac_create(grid, horizon=None, rho=None, params=None, stream=0):
    return ucac_create_batch([grid], None if horizon is None else [horizon], None if rho is None else [rho],
                             params, stream)


def ucac_instances(h) -> int:
    return lib().ucac_instances(h)


def ucac_iterate(h, n_sweeps: int) -> int:
    return _check(lib().ucac_iterate(h, int(n_sweeps)), h)


def ucac_enqueue_sweeps(h, n_sweeps: int) -> int:
    return _check(lib().ucac_enqueue_sweeps(h, int(n_sweeps)), h)


def ucac_residuals(h, instance: int = 0) -> dict:
    r = ucac_report()
    _check(lib().ucac_residuals(h, int(instance), C.byref(r)), h)
    return {f: getattr(r, f) for f, _ in ucac_report._fields_}


def solution_arrays(T: int, ng: int, nb: int, nl: int, alloc=np.zeros) -> dict:
    """Output arrays of ucac_solution for one instance (alloc(shape, dtype),
    e.g. a page-locked allocator)."""
    return {"p": alloc((T, ng), np.float64), "q": alloc((T, ng), np.float64), "w": alloc((T, nb), np.float64),
            "theta": alloc((T, nb), np.float64), "pf": alloc((T, nl, 4), np.float64),
            "u_on": alloc((T, ng), np.uint8)}


def ucac_solution(h, instance: int, T: int, ng: int, nb: int, nl: int, out: dict | None = None) -> dict:
    """The instance's solution; out: arrays from solution_arrays to fill
    (C-contiguous, of those shapes and dtypes), else new ones."""
    o = solution_arrays(T, ng, nb, nl) if out is None else out
    for name, shape, dt in (("p", (T, ng), np.float64), ("q", (T, ng), np.float64), ("w", (T, nb), np.float64),
                            ("theta", (T, nb), np.float64), ("pf", (T, nl, 4), np.float64),
                            ("u_on", (T, ng), np.uint8)):
        a = o[name]
        if a.shape != shape or a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise UcacError(f"solution array {name}: expected {shape} {np.dtype(dt)} C-contiguous")
    p, q, w, th, pf, u = o["p"], o["q"], o["w"], o["theta"], o["pf"], o["u_on"]
    _check(lib().ucac_solution(h, int(instance), p.ctypes.data_as(_dp), q.ctypes.data_as(_dp), w.ctypes.data_as(_dp),
                               th.ctypes.data_as(_dp), pf.ctypes.data_as(_dp),
                               u.ctypes.data_as(C.POINTER(C.c_uint8))), h)
    return o


def ucac_line_counts(h, instance: int, T: int, nl: int) -> tuple:
    """Newton iterations and multiplier rounds of each line-period's solve in
    the last sweep the instance ran, two [T][n_branch] uint16 arrays."""
    nw = np.zeros((T, nl), np.uint16)
    na = np.zeros((T, nl), np.uint16)
    _check(lib().ucac_line_counts(h, int(instance), nw.ctypes.data_as(C.POINTER(C.c_uint16)),
                                  na.ctypes.data_as(C.POINTER(C.c_uint16))), h)
    return nw, na


def count_histogram(counts: np.ndarray, top: int = 8) -> list:
    """Histogram of per-solve counts: bins 0 .. top - 1 and a last bin for
    top or more."""
    c = np.minimum(np.asarray(counts).ravel().astype(np.int64), top)
    return np.bincount(c, minlength=top + 1).tolist()


def ucac_state_size(h, instance: int = 0) -> int:
    return int(lib().ucac_state_size(h, int(instance)))


def ucac_state_export(h, instance: int = 0) -> np.ndarray:
    n = ucac_state_size(h, instance)
    buf = np.empty(n, np.float64)
    _check(lib().ucac_state_export(h, int(instance), buf.ctypes.data_as(_dp), n), h)
    return buf


def ucac_state_import(h, instance: int, buf: np.ndarray) -> None:
    buf = np.ascontiguousarray(buf, np.float64)
    _check(lib().ucac_state_import(h, int(instance), buf.ctypes.data_as(_dp), buf.size), h)


def ucac_kernel_times(h, n_sweeps: int = 5) -> dict:
    ms = np.zeros(UCAC_N_KERNELS)
    _check(lib().ucac_kernel_times(h, int(n_sweeps), ms.ctypes.data_as(_dp)), h)
    return {ucac_kernel_name(k): float(ms[k]) for k in range(UCAC_N_KERNELS)}


def ucac_kernel_name(k: int) -> str:
    return lib().ucac_kernel_name(int(k)).decode()


def ucac_ucdp_workspace_bytes(n_gen: int, T: int) -> int:
    return int(lib().ucac_ucdp_workspace_bytes(int(n_gen), int(T)))


def ucac_ucdp(n_gen, T, rho_uc, tau_on, tau_su, tau_sd, c0, c_su, c_sd, TU, TD, u0, K0, u_on, cost, workspace,
              workspace_bytes, stream=0):
    """All array arguments are device pointers (ints), e.g. torch_tensor.data_ptr()."""
    vp = C.c_void_p
    return _check(lib().ucac_ucdp(int(n_gen), int(T), float(rho_uc), *[vp(int(x)) for x in
                                  (tau_on, tau_su, tau_sd, c0, c_su, c_sd, TU, TD, u0, K0, u_on, cost)],
                                  vp(int(workspace)), int(workspace_bytes), vp(int(stream))))


UCAC_UCDP_NOALLOC_MAX_BYTES = 16 << 20


def ucac_ucdp_noalloc(n_gen, T, rho_uc, tau_on, tau_su, tau_sd, c0, c_su, c_sd, TU, TD, u0, K0, u_on, cost, stream=0):
    """Same as ucac_ucdp without a workspace (library-owned static scratch); device pointers as ints."""
    vp = C.c_void_p
    return _check(lib().ucac_ucdp_noalloc(int(n_gen), int(T), float(rho_uc), *[vp(int(x)) for x in
                                          (tau_on, tau_su, tau_sd, c0, c_su, c_sd, TU, TD, u0, K0, u_on, cost)],
                                          vp(int(stream))))


def ucac_probe_fp64(reps: int = 5, stream=0) -> float:
    f = C.c_double()
    _check(lib().ucac_probe_fp64(int(reps), C.c_void_p(stream), C.byref(f)))
    return f.value


def ucac_probe_cossin(d) -> tuple:
    """The polar line kernel's cos/sin of the angles d (|d| <= pi), on the device."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    c, s = np.empty_like(d), np.empty_like(d)
    _check(lib().ucac_probe_cossin(int(d.size), d.ctypes.data_as(_dp), c.ctypes.data_as(_dp), s.ctypes.data_as(_dp)))
    return c, s


def ucac_probe_dw(op: int, x, y=None, z=None):
    """One double-word operation of the line kernel's evaluation on the
    device (see include/ucac.h): an (n, 4) array of result parts."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x) if y is None else np.ascontiguousarray(y, dtype=np.float64)
    z = np.zeros_like(x) if z is None else np.ascontiguousarray(z, dtype=np.float64)
    out = np.zeros((x.size, 4))
    _check(lib().ucac_probe_dw(int(op), int(x.size), x.ctypes.data_as(_dp), y.ctypes.data_as(_dp),
                               z.ctypes.data_as(_dp), out.ctypes.data_as(_dp)))
    return out


def ucac_autotune(h, sweeps_per_trial: int = 3, cache_path: str | None = None) -> dict:
    out = np.zeros(5, np.int32)
    cp = cache_path.encode() if cache_path else None
    _check(lib().ucac_autotune(h, int(sweeps_per_trial), cp, out.ctypes.data_as(_ip)), h)
    return dict(zip(("ucdp", "gen", "line", "bus", "ucbar"), (int(v) for v in out)))


def ucac_uc_warm_start(h, relax_sweeps: int = 300, p_frac: float = 0.5) -> None:
    _check(lib().ucac_uc_warm_start(h, int(relax_sweeps), float(p_frac)), h)


def ucac_mlp_param_count() -> int:
    return int(lib().ucac_mlp_param_count())


def ucac_mlp_workspace_bytes(n: int) -> int:
    return int(lib().ucac_mlp_workspace_bytes(int(n)))


def ucac_mlp_forward(n, params, x, y, workspace, workspace_bytes, stream=0):
    """Tensor-core inference on DEVICE pointers (ints); synchronises."""
    _check(lib().ucac_mlp_forward(int(n), params, x, y, workspace, int(workspace_bytes), stream))


def ucac_mlp_grad(n, params, x, labels, grad, loss, workspace, workspace_bytes, stream=0):
    """FP32 loss and gradient on DEVICE pointers (ints); enqueued."""
    _check(lib().ucac_mlp_grad(int(n), params, x, labels, grad, loss, workspace, int(workspace_bytes), stream))


def ucac_mlp_adam(params, grad, m, v, step, lr, stream=0):
    _check(lib().ucac_mlp_adam(params, grad, m, v, int(step), float(lr), stream))


def ucac_line_features(h, instance: int, n_rows: int):
    """(features [n_rows][12] float32, residual norms [n_rows] float64) of the
    instance's line-periods (n_rows = horizon * n_branch) at the current iterate."""
    f = np.zeros((n_rows, 12), np.float32)
    sc = np.zeros(n_rows)
    _check(lib().ucac_line_features(h, int(instance), f.ctypes.data_as(C.POINTER(C.c_float)), sc.ctypes.data_as(_dp)),
           h)
    return f, sc


def ucac_line_samples(h, n_rows: int, features=True, iterate=True):
    """(features [n][12] float32 or None, norms [n] or None, W iterates [n][6] or None)
    of all line-periods of the handle (n_rows = sum of horizon * n_branch)."""
    f = np.zeros((n_rows, 12), np.float32) if features else None
    sc = np.zeros(n_rows) if features else None
    x = np.zeros((n_rows, 6)) if iterate else None
    _check(lib().ucac_line_samples(h, f.ctypes.data_as(C.POINTER(C.c_float)) if features else None,
                                   sc.ctypes.data_as(_dp) if features else None,
                                   x.ctypes.data_as(_dp) if iterate else None), h)
    return f, sc, x


def ucac_set_warm_start(h, params) -> None:
    if params is None:
        _check(lib().ucac_set_warm_start(h, None), h)
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != ucac_mlp_param_count():
        raise UcacError(f"warm-start parameters: expected {ucac_mlp_param_count()} values, got {p.size}")
    _check(lib().ucac_set_warm_start(h, p.ctypes.data_as(C.POINTER(C.c_float))), h)


def ucac_set_warmstart(h, blob_bf16) -> None:
    """The network as BF16 bit patterns (uint16 array of ucac_mlp_param_count()
    values), or None to disable the learned start."""
    if blob_bf16 is None:
        _check(lib().ucac_set_warmstart(h, None, 0), h)
        return
    b = np.ascontiguousarray(blob_bf16, dtype=np.uint16)
    _check(lib().ucac_set_warmstart(h, C.c_void_p(b.ctypes.data), b.nbytes), h)


def ucac_warm_start_stats(h, instance: int = 0):
    taken = C.c_int64(0)
    err = C.c_int32(0)
    _check(lib().ucac_warm_start_stats(h, int(instance), C.byref(taken), C.byref(err)), h)
    return int(taken.value), int(err.value)


def ucac_destroy(h) -> None:
    if h:
        lib().ucac_destroy(h)


def ucac_last_error(h=None) -> str:
    m = lib().ucac_last_error(h)
    return m.decode() if m else ""


class Handle:
    """RAII wrapper: a batch of instances on the current CUDA device."""

    def __init__(self, grids, params=None, stream=0, horizons=None):
        self.grids = list(grids)
        self.horizons = list(horizons) if horizons is not None else None
        self.h = ucac_create_batch(self.grids, horizons=horizons, params=params, stream=stream)

    def close(self):
        if getattr(self, "h", None):
            ucac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, n):
        return ucac_iterate(self.h, n)

    def enqueue(self, n):
        return ucac_enqueue_sweeps(self.h, n)

    def residuals(self, k=0):
        return ucac_residuals(self.h, k)

    def line_counts(self, k=0):
        T = self.horizons[k] if self.horizons is not None else self.grids[k].T
        return ucac_line_counts(self.h, k, T, self.grids[k].n_branch)

    def export(self, k=0):
        return ucac_state_export(self.h, k)

    def import_(self, k, buf):
        ucac_state_import(self.h, k, buf)

    def kernel_times(self, n=5):
        return ucac_kernel_times(self.h, n)

    def autotune(self, sweeps_per_trial=3, cache_path=None):
        return ucac_autotune(self.h, sweeps_per_trial, cache_path)

    def line_features(self, k=0):
        T = self.horizons[k] if self.horizons is not None else self.grids[k].T
        return ucac_line_features(self.h, k, T * self.grids[k].n_branch)

    def uc_warm_start(self, relax_sweeps=300, p_frac=0.5):
        ucac_uc_warm_start(self.h, relax_sweeps, p_frac)

    def line_rows(self):
        return sum((self.horizons[k] if self.horizons is not None else g.T) * g.n_branch
                   for k, g in enumerate(self.grids))

    def line_samples(self, features=True, iterate=True):
        return ucac_line_samples(self.h, self.line_rows(), features, iterate)

    def set_warm_start(self, params):
        ucac_set_warm_start(self.h, params)

    def warm_start_stats(self, k=0):
        return ucac_warm_start_stats(self.h, k)
