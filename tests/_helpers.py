"""Shared helpers of the tests: state comparison in the canonical layout."""
import numpy as np

import oracle

# UC decisions and counters are compared bit for bit.
EXACT_FIELDS = {"u_on", "u_su", "u_sd", "l_inner", "k_outer", "pending", "done", "rho_pq", "rho_va", "rho_uc",
                "rho_cnt", "rho_log"}
# Per-iterate bound of the FP64 path against the oracle: normwise relative
# 1e-9 per field, plus an absolute floor at the FP64 noise level of the
# quantity (positions and powers are O(1) p.u.; multipliers y carry a factor
# rho; the line multipliers mu are known only up to c * eps_mach, since the
# augmented-Lagrangian update mu += c h multiplies the rounding of h by c).
RTOL = 1e-9
ATOL = 1e-12


def field_atol(name, g, cpen_max, mu_eta=None):
    rho_pq, rho_va, rho_uc = g.rho
    if name.startswith("gy_") or name.startswith("glam_"):
        r = name.split("_", 1)[1]
        return ATOL * (rho_uc if r in ("on", "su", "sd") else rho_pq)
    if name.startswith("by_") or name.startswith("blam_"):
        r = name.split("_", 1)[1]
        return ATOL * (rho_pq if r in ("pij", "qij", "pji", "qji") else rho_va)
    if name.startswith("mu"):
        # a solver that reaches the line subproblem's KKT point by another
        # path (mu_eta = its stopping tolerance eta on |h|) fixes mu = mu + c h
        # only to within c eta on each side
        return (2.0 * mu_eta if mu_eta is not None else 1e-14) * cpen_max
    if name in ("beta", "beta_next", "zprev"):
        return 0.0
    return ATOL


def compare_states(a, b, g, rtol=RTOL, skip=(), mu_eta=None):
    """Returns a list of (field, err, bound) that violate the bound."""
    dims = (g.T, g.n_gen, g.n_branch, g.n_bus)
    A = oracle.unpack_state(a, *dims)
    B = oracle.unpack_state(b, *dims)
    cmax = max(float(np.abs(A["cpen"]).max()), float(np.abs(B["cpen"]).max()))
    bad = []
    for name in A:
        if name in skip:
            continue
        x, y = np.asarray(A[name], float), np.asarray(B[name], float)
        if name in EXACT_FIELDS:
            if not np.array_equal(x, y):
                bad.append((name, float(np.abs(x - y).max()), 0.0))
            continue
        err = float(np.abs(x - y).max()) if x.size else 0.0
        scale = max(float(np.abs(x).max()) if x.size else 0.0, float(np.abs(y).max()) if y.size else 0.0)
        bound = rtol * scale + field_atol(name, g, cmax, mu_eta)
        if not err <= bound:
            bad.append((name, err, bound))
    return bad
