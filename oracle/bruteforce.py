"""Brute-force UC enumeration (TEST INFRASTRUCTURE ONLY).

Independent of the dynamic program: it enumerates every on/off schedule,
derives start-ups and shut-downs as su_t = max(0, u_t - u_{t-1}),
sd_t = max(0, u_{t-1} - u_t) (Sec. III-B), keeps the schedules that satisfy
the UC_g constraints exactly as written in Eq. set:UC (initial forced periods,
minimum up and down windows), and evaluates the augmented-Lagrangian UC
objective of Eq. step:uc in its original form
  sum_t c0 u_t + c_su su_t + c_sd sd_t
        + sum_k y_k (u_k - ubar_k + z_k) + rho/2 (u_k - ubar_k + z_k)^2 .
"""
from __future__ import annotations

import itertools

import numpy as np


def derived(u, u0):
    """(su, sd) from an on/off schedule and the period-0 status."""
    prev = np.concatenate([[u0], u[:-1]])
    return np.maximum(0, u - prev), np.maximum(0, prev - u)


def feasible(u, u0, L, F, TU, TD):
    """Eq. uc_initial_on/off, uc_minup, uc_mindn (1-based t in the paper)."""
    u = np.asarray(u, dtype=np.int64)
    T = u.size
    su, sd = derived(u, u0)
    if L > 0 and np.sum(1 - u[:L]) != 0:
        return False
    if F > 0 and np.sum(u[:F]) != 0:
        return False
    for t in range(TU, T + 1):  # t = TU..T
        if su[t - TU:t].sum() > u[t - 1]:
            return False
    for t in range(TD, T + 1):
        if sd[t - TD:t].sum() > 1 - u[t - 1]:
            return False
    return True


def objective(u, u0, c0, csu, csd, rho, ubar, y, z):
    """ubar, y, z: arrays [3][T] for the rows (on, su, sd)."""
    u = np.asarray(u, dtype=np.float64)
    su, sd = derived(u, u0)
    x = np.stack([u, su, sd])
    r = x - ubar + z
    return float(np.sum(c0 * u + csu * su + csd * sd) + np.sum(y * r) + 0.5 * rho * np.sum(r * r))


def best_schedule(T, u0, L, F, TU, TD, c0, csu, csd, rho, ubar, y, z):
    best, arg = np.inf, None
    for bits in itertools.product((0, 1), repeat=T):
        u = np.array(bits)
        if not feasible(u, u0, L, F, TU, TD):
            continue
        f = objective(u, u0, c0, csu, csd, rho, ubar, y, z)
        if f < best:
            best, arg = f, u
    return best, arg
