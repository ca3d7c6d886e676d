"""Shared helpers of the tests: state comparison in the canonical layout."""
import json
import os

import numpy as np

import oracle

# UC decisions and counters are compared bit for bit.
EXACT_FIELDS = {"u_on", "u_su", "u_sd", "l_inner", "k_outer", "pending", "done", "rho_pq", "rho_va", "rho_uc",
                "rho_cnt", "rho_log"}
# Per-iterate bound of the FP64 path against the oracle, element by element:
#   |gpu_i - ref_i| <= RTOL |ref_i| + floor_i
# and, beside it, the normwise form |gpu_i - ref_i| <= RTOL max|ref| + floor_i.
# The floor is the noise level of the quantity in absolute terms (p.u.; a
# multiplier y or lambda carries a factor rho):
#  - ATOL = 1e-12 for the generator-side and UC fields, which both sides
#    compute in closed form or by exact enumeration (FP64 rounding only);
#  - ATOL_LINE = 5e-11 for everything the line subproblems feed (their
#    variables, flows and rows, the bus copies and the generator consensus
#    rows coupled to them through the bus projection): a line solve is fixed
#    only up to its stopping rule (reading R6: the last step is below
#    1e-9 (1 + |x|), and the Newton step that follows it would be smaller by
#    the contraction of the step, up to cond(H) 2^-24 ~ 6e-4 with the FP32
#    Hessian, i.e. ~1.2e-12 in V), and the flows multiply that by the line
#    admittance (|y| <= 20 p.u.) at both ends;
#  - a line-limit multiplier mu is known only up to its own line's penalty c
#    times the rounding of h (1e-14 c), or, for a solver that reaches the line
#    subproblem's KKT point by another path with the inner stopping tolerance
#    eta on |h|, up to 2 c eta (each side fixes mu = mu + c h within c eta).
RTOL = 1e-9
ATOL = 1e-12
ATOL_LINE = 5e-11
LINE_COUPLED = ("v", "fb", "by_", "bz_", "blam_", "wbar", "thbar", "pbar", "qbar", "gy_gp", "gy_gq", "gy_tc",
                "gz_gp", "gz_gq", "gz_tc", "glam_gp", "glam_gq", "glam_tc")

# Achieved errors per (test, field), written to $UCAC_PARITY_LOG at the end
# of the session when that variable is set (see conftest.py).
STATS = {}


def field_floor(name, g, cpen, mu_eta=None):
    """Absolute floor of one field: a scalar, or an array for mu (per line-period)."""
    rho_pq, rho_va, rho_uc = g.rho
    if name.startswith("mu"):
        return (2.0 * mu_eta if mu_eta is not None else 1e-14) * cpen
    if name in ("beta", "beta_next", "zprev"):
        return 0.0
    a = ATOL_LINE if name.startswith(LINE_COUPLED) else ATOL
    if name.startswith("gy_") or name.startswith("glam_"):
        r = name.split("_", 1)[1]
        return a * (rho_uc if r in ("on", "su", "sd") else rho_pq)
    if name.startswith("by_") or name.startswith("blam_"):
        r = name.split("_", 1)[1]
        return a * (rho_pq if r in ("pij", "qij", "pji", "qji") else rho_va)
    return a


def compare_states(a, b, g, rtol=RTOL, skip=(), mu_eta=None, label=None):
    """a = library iterate, b = oracle iterate (the reference), both in the
    canonical layout.  Returns a list of (field, err, bound, kind) for every
    field that violates the element-wise or the normwise bound."""
    if label is None:
        label = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0] or None
    dims = (g.T, g.n_gen, g.n_branch, g.n_bus)
    A = oracle.unpack_state(a, *dims)
    B = oracle.unpack_state(b, *dims)
    cpen = np.maximum(np.abs(np.asarray(A["cpen"], float)), np.abs(np.asarray(B["cpen"], float)))
    bad = []
    for name in A:
        if name in skip:
            continue
        x, y = np.asarray(A[name], float), np.asarray(B[name], float)
        if name in EXACT_FIELDS:
            if not np.array_equal(x, y):
                bad.append((name, float(np.abs(x - y).max()), 0.0, "exact"))
            continue
        if x.size == 0:
            continue
        err = np.abs(x - y)
        floor = field_floor(name, g, cpen, mu_eta)
        scale = float(np.abs(y).max())
        if label is not None:
            # achieved errors: normwise relative, element-wise relative over
            # the elements above the floor's level, and absolute
            big = np.abs(y) * rtol > floor
            erel = float((err[big] / np.abs(y[big])).max()) if np.any(big) else 0.0
            s = STATS.setdefault(label, {}).setdefault(name, [0.0, 0.0, 0.0])
            s[0] = max(s[0], float(err.max()) / scale if scale > 0 else float(err.max()))
            s[1] = max(s[1], erel)
            s[2] = max(s[2], float(err.max()))
        # element-wise: each element against its own reference value
        lim_e = rtol * np.abs(y) + floor
        if not np.all(err <= lim_e):
            i = int(np.argmax(err - lim_e))
            bad.append((name, float(np.ravel(err)[i]), float(np.ravel(lim_e * np.ones_like(err))[i]), "elem"))
            continue
        # normwise: against the largest reference value of the field
        lim_n = rtol * scale + floor
        if not np.all(err <= lim_n):
            bad.append((name, float(err.max()), float(np.max(lim_n)), "norm"))
    return bad


def dump_stats():
    path = os.environ.get("UCAC_PARITY_LOG")
    if path and STATS:
        with open(path, "w") as f:
            json.dump(STATS, f, indent=1, sort_keys=True)
