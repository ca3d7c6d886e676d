"""FP64 CPU oracle for the UC-ACOPF component-ADMM sweep.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke entry point and the
benchmark's CPU-baseline leg may import this package.  The CUDA library never
loads it, and this package never loads the CUDA library: they share nothing
but the raw grid arrays drawn by the seeded input generator.

The arithmetic lives in plain C (`ucac_oracle.c`); this module builds it with
gcc and wraps it with ctypes.  Parity status of each routine is listed in the
C file's header comments; every routine is pinned by `-m "not gpu"` tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off: every op rounded
    separately); omp=True builds the OpenMP variant (the x-step subproblems
    on all host cores, the same bits)."""
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] + (["-fopenmp"] if omp else [])
                              + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class OrcGrid(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("n_gen", C.c_int32), ("T", C.c_int32),
                ("ref_bus", C.c_int32)] + \
        [(n, _dp) for n in ("Pd", "Qd", "Gs", "Bs", "Vmin", "Vmax")] + \
        [(n, _ip) for n in ("br_from", "br_to")] + \
        [(n, _dp) for n in ("br_r", "br_x", "br_b", "br_rate")] + \
        [("gen_bus", _ip)] + \
        [(n, _dp) for n in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0", "c_su", "c_sd", "RU", "RD", "SU", "SD")] + \
        [(n, _ip) for n in ("TU", "TD", "u0", "L0", "F0")] + \
        [("p0", _dp), ("base_mva", C.c_double)]


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rho_pq", "rho_va", "rho_uc", "eps_in", "eps_out", "tau", "theta",
                                          "beta0", "lam_max", "eta", "omega_rel", "c_init_rel", "c_max_rel",
                                          "rho_mu", "rho_tau")] + \
        [(n, C.c_int32) for n in ("K_AL", "K_N", "L_max", "uc_relax", "rho_every", "pad")]


def lib(omp: bool = False):
    """The plain build (default) or the OpenMP build; the same entry points."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            L = C.CDLL(build(omp=omp))
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(OrcGrid), C.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_state_size.restype = C.c_long
            L.orc_state_size.argtypes = [C.c_void_p]
            L.orc_state_get.argtypes = [C.c_void_p, _dp]
            L.orc_state_set.argtypes = [C.c_void_p, _dp]
            L.orc_sweep.argtypes = [C.c_void_p]
            L.orc_residuals.argtypes = [C.c_void_p, _dp, C.POINTER(C.c_long)]
            L.orc_rows.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_default_params.argtypes = [C.POINTER(OrcParams)]
            L.orc_uc_stagecost.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
            L.orc_dp.restype = C.c_double
            L.orc_dp.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _ip]
            L.orc_gen_solve.argtypes = [_dp, C.c_int, _dp, _dp]
            L.orc_branch_solve.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_int, C.c_int, _dp, _dp, _dp, _dp, _ip]
            L.orc_bus_solve.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
            L.orc_boxqp.argtypes = [C.c_int, _dp, _dp, _dp]
            L.orc_ucdp_batch.argtypes = [C.c_int, C.c_int, C.c_double] + [_dp] * 6 + [_ip] * 4 + \
                [C.POINTER(C.c_int8), _dp]
            L.orc_threads.argtypes = [C.c_int]
            L.orc_threads.restype = C.c_int
            if omp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if omp else _lib


def threads(n: int = 0) -> int:
    """Sets (n > 0) and returns the thread count of the OpenMP build."""
    return lib(omp=True).orc_threads(int(n))


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def default_params(rho=None, **kw) -> OrcParams:
    p = OrcParams()
    lib().orc_default_params(C.byref(p))
    if rho is not None:
        p.rho_pq, p.rho_va, p.rho_uc = (float(v) for v in rho)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- state layout
GEN_FIELDS = ["p", "q", "ph", "s_pl", "s_pu", "s_ql", "s_qu", "s_rd", "s_ru", "u_on", "u_su", "u_sd",
              "pbar", "qbar", "ub_on", "ub_su", "ub_sd"]
GEN_ROWS = ["on", "su", "sd", "pl", "pu", "ql", "qu", "rd", "ru", "gp", "gq", "tc"]
BR_FIELDS = ["v%d" % k for k in range(8)] + ["mu%d" % k for k in range(4)] + ["cpen"] + ["fb%d" % k for k in range(4)]
BR_ROWS = ["pij", "qij", "pji", "qji", "wi", "wj", "thi", "thj"]
BUS_FIELDS = ["wbar", "thbar"]
CTRL = ["beta", "zprev", "l_inner", "k_outer", "pending", "beta_next", "done", "rho_pq", "rho_va", "rho_uc",
        "rho_cnt", "rho_log"]


def state_layout(T, ng, nl, nb):
    """(name, shape) in the canonical order shared by the oracle and the library's export."""
    out = [(f, (T, ng)) for f in GEN_FIELDS]
    for kind in ("y", "z", "lam"):
        out += [("g%s_%s" % (kind, r), (T, ng)) for r in GEN_ROWS]
    out += [(f, (T, nl)) for f in BR_FIELDS]
    for kind in ("y", "z", "lam"):
        out += [("b%s_%s" % (kind, r), (T, nl)) for r in BR_ROWS]
    out += [(f, (T, nb)) for f in BUS_FIELDS]
    out += [(c, ()) for c in CTRL]
    return out


def unpack_state(buf, T, ng, nl, nb):
    st, o = {}, 0
    for name, shp in state_layout(T, ng, nl, nb):
        n = int(np.prod(shp)) if shp else 1
        st[name] = buf[o:o + n].reshape(shp) if shp else float(buf[o])
        o += n
    assert o == buf.size
    return st


def pack_state(st, T, ng, nl, nb):
    parts = []
    for name, shp in state_layout(T, ng, nl, nb):
        parts.append(np.asarray(st[name], dtype=np.float64).reshape(-1) if shp else np.array([st[name]], np.float64))
    return np.ascontiguousarray(np.concatenate(parts))


# ---------------------------------------------------------------- instances
class Oracle:
    """One instance of the sweep on the CPU (plain FP64).  omp=True runs it on
    the OpenMP build (x-step subproblems on all host cores, the same bits)."""

    def __init__(self, grid, params: OrcParams | None = None, omp: bool = False, **kw):
        L = self._L = lib(omp)
        self.grid = grid
        self.params = params if params is not None else default_params(rho=grid.rho, **kw)
        self._keep = []

        def dd(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return _d(a)

        def ii(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self._keep.append(a)
            return _i(a)

        g = grid
        s = OrcGrid()
        s.n_bus, s.n_branch, s.n_gen, s.T, s.ref_bus = g.n_bus, g.n_branch, g.n_gen, g.T, g.ref_bus
        for n in ("Pd", "Qd", "Gs", "Bs", "Vmin", "Vmax", "br_r", "br_x", "br_b", "br_rate", "Pmin", "Pmax", "Qmin",
                  "Qmax", "c2", "c1", "c0", "c_su", "c_sd", "RU", "RD", "SU", "SD", "p0"):
            setattr(s, n, dd(getattr(g, n)))
        for n in ("br_from", "br_to", "gen_bus", "TU", "TD", "u0", "L0", "F0"):
            setattr(s, n, ii(getattr(g, n)))
        s.base_mva = g.base_mva
        self._s = s
        h = L.orc_create(C.byref(s), C.byref(self.params))
        if not h:
            raise ValueError("oracle rejected the grid data")
        self._h = C.c_void_p(h)
        self.dims = (g.T, g.n_gen, g.n_branch, g.n_bus)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_L", None) is not None:
            self._L.orc_destroy(h)
            self._h = None

    def state_vector(self):
        L = self._L
        buf = np.empty(L.orc_state_size(self._h), np.float64)
        L.orc_state_get(self._h, _d(buf))
        return buf

    def state(self):
        return unpack_state(self.state_vector(), *self.dims)

    def set_state(self, st):
        buf = st if isinstance(st, np.ndarray) else pack_state(st, *self.dims)
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        assert buf.size == self._L.orc_state_size(self._h)
        self._L.orc_state_set(self._h, _d(buf))

    def sweep(self, n: int = 1):
        for _ in range(n):
            self._L.orc_sweep(self._h)

    def residuals(self):
        out = np.zeros(6)
        st = (C.c_long * 4)()
        self._L.orc_residuals(self._h, _d(out), st)
        keys = ("r_p", "r_d", "z_norm", "inf_norm", "objective", "z_rms")
        d = {k: float(v) for k, v in zip(keys, out)}
        d.update(sweeps=st[0], newton=st[1], al=st[2], branch_fail=st[3])
        return d

    def rows(self):
        T, ng, nl, nb = self.dims
        GA = np.zeros((12, T, ng)); GB = np.zeros((12, T, ng))
        BA = np.zeros((8, T, nl)); BB = np.zeros((8, T, nl))
        self._L.orc_rows(self._h, _d(GA), _d(GB), _d(BA), _d(BB))
        return GA, GB, BA, BB


# ---------------------------------------------------------------- components
def uc_stagecost(c0, csu, csd, rho, tau_on, tau_su, tau_sd):
    tau_on, tau_su, tau_sd = (np.ascontiguousarray(x, np.float64) for x in (tau_on, tau_su, tau_sd))
    T = tau_on.size
    L = np.zeros((T, 4))
    lib().orc_uc_stagecost(T, c0, csu, csd, rho, _d(tau_on), _d(tau_su), _d(tau_sd), _d(L))
    return L


def dp(L, TU, TD, u0, K0=0):
    """Algorithm 2 on a stage-cost table L[t][a*2+b]; returns (cost, u_on)."""
    L = np.ascontiguousarray(L, np.float64)
    T = L.shape[0]
    u = np.zeros(T, np.int32)
    c = lib().orc_dp(T, int(TU), int(TD), int(u0), int(K0), _d(L), _i(u))
    return c, u


def ucdp_batch(rho, tau_on, tau_su, tau_sd, c0, csu, csd, TU, TD, u0, K0):
    """Algorithm 2 for every generator of [T][n_gen] inputs; returns (u_on int8 [T][n_gen], cost [n_gen])."""
    tau_on, tau_su, tau_sd, c0, csu, csd = (np.ascontiguousarray(x, np.float64)
                                            for x in (tau_on, tau_su, tau_sd, c0, csu, csd))
    TU, TD, u0, K0 = (np.ascontiguousarray(x, np.int32) for x in (TU, TD, u0, K0))
    T, ng = tau_on.shape
    u = np.zeros((T, ng), np.int8)
    cost = np.zeros(ng)
    lib().orc_ucdp_batch(ng, T, float(rho), _d(tau_on), _d(tau_su), _d(tau_sd), _d(c0), _d(csu), _d(csd), _i(TU),
                         _i(TD), _i(u0), _i(K0), u.ctypes.data_as(C.POINTER(C.c_int8)), _d(cost))
    return u, cost


def gen_solve(prm, has_prev, tg):
    prm = np.ascontiguousarray(prm, np.float64)
    tg = np.ascontiguousarray(tg, np.float64)
    out = np.zeros(9)
    lib().orc_gen_solve(_d(prm), int(has_prev), _d(tg), _d(out))
    return out


def branch_solve(cst, tgt, rho_pq, rho_va, v, mu, c, eta=1e-12, omega=None, c_max=None, K_AL=50, K_N=50):
    cst = np.ascontiguousarray(cst, np.float64)
    tgt = np.ascontiguousarray(tgt, np.float64)
    v = np.array(v, np.float64)
    mu = np.array(mu, np.float64)
    cc = np.array([c], np.float64)
    a = np.zeros(8)
    info = np.zeros(3, np.int32)
    rmax = max(rho_pq, rho_va)
    omega = 1e-12 * rmax if omega is None else omega
    c_max = 1e6 * rmax if c_max is None else c_max
    lib().orc_branch_solve(_d(cst), _d(tgt), rho_pq, rho_va, eta, omega, c_max, K_AL, K_N, _d(v), _d(mu), _d(cc),
                           _d(a), _i(info))
    return v, mu, float(cc[0]), a, info


def bus_solve(W, m, aP, aQ, Pd, Qd):
    W, m, aP, aQ = (np.ascontiguousarray(x, np.float64) for x in (W, m, aP, aQ))
    v = np.zeros(W.size)
    lib().orc_bus_solve(W.size, _d(W), _d(m), _d(aP), _d(aQ), float(Pd), float(Qd), _d(v))
    return v


def boxqp(H, g):
    H = np.ascontiguousarray(H, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    x = np.zeros(g.size)
    lib().orc_boxqp(g.size, _d(H.reshape(-1)), _d(g), _d(x))
    return x
