"""Seeded synthetic UC-ACOPF instances.

This module only draws input data (grid topology, line parameters, loads,
generator data).  It holds none of the method's arithmetic: admittances,
coupling rows, cold start and every ADMM step are computed separately by the
CUDA library and by the CPU oracle, each from the raw data produced here.

The shapes follow the paper's workloads (Sec. IV "Test Instances"): hourly
periods, a daily load shape discounted by 0.7 so that some units can be
switched off, quadratic generation costs, ramp limits and 2 h minimum up/down
times.  The MATPOWER cases and ISO-NE load series the paper uses are not
reproduced; seeded random grids of the same kind stand in for them.

All randomness comes from numpy's counter-based Philox generator, keyed by
(seed, stream) so that each data family has its own reproducible stream.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

__all__ = ["Grid", "make_grid", "config_instances", "CONFIGS", "RHO_TABLE"]

# Random networks drawn here are far weaker than MATPOWER's (per-bus loads
# U(0.5,1.5) p.u. against 1-3 p.u. line ratings and reactances up to 0.3 p.u.);
# at the configured load level most draws are AC-infeasible (voltage lower
# bounds and generator reactive limits bind at the far end of long radial
# paths, and the ADMM stalls with |Ax + Bxbar|_inf ~ 0.1).  Every load is
# therefore multiplied by a network-loading factor on top of the paper's 0.7
# discount: 0.4 up to 300 buses, decreasing as (300/n)^(1/4) beyond (0.25 at
# 2000 buses), since path lengths grow with the size of the random grid.
NETWORK_LOADING = 0.4


def network_loading(n_bus: int) -> float:
    return NETWORK_LOADING * min(1.0, (300.0 / n_bus) ** 0.25)


# Penalties per workload, taken from the paper's Table 1 rows (case9 for the
# 9-bus grid, case118 for the 118-bus grid, case300 for the large ones).
RHO_TABLE = {
    "case9": (5e3, 1e4, 1e4),
    "case118": (5e4, 1e5, 1e5),
    "case300": (5e3, 1e4, 1e4),
}


@dataclasses.dataclass
class Grid:
    """One UC-ACOPF instance in SoA form (0-based indices, per-unit, FP64)."""

    n_bus: int
    n_branch: int
    n_gen: int
    T: int
    ref_bus: int
    Pd: np.ndarray  # [T][n_bus]
    Qd: np.ndarray  # [T][n_bus]
    Gs: np.ndarray  # [n_bus]
    Bs: np.ndarray
    Vmin: np.ndarray
    Vmax: np.ndarray
    br_from: np.ndarray  # int32 [n_branch]
    br_to: np.ndarray
    br_r: np.ndarray
    br_x: np.ndarray
    br_b: np.ndarray
    br_rate: np.ndarray
    gen_bus: np.ndarray  # int32 [n_gen]
    Pmin: np.ndarray
    Pmax: np.ndarray
    Qmin: np.ndarray
    Qmax: np.ndarray
    c2: np.ndarray  # $/MW^2 h
    c1: np.ndarray  # $/MWh
    c0: np.ndarray  # $/h when on
    c_su: np.ndarray  # $ per start-up
    c_sd: np.ndarray  # $ per shut-down
    RU: np.ndarray  # p.u. per period
    RD: np.ndarray
    SU: np.ndarray
    SD: np.ndarray
    TU: np.ndarray  # int32 periods
    TD: np.ndarray
    u0: np.ndarray  # int32 0/1
    L0: np.ndarray  # int32 forced-on periods at the start
    F0: np.ndarray  # int32 forced-off periods at the start
    p0: np.ndarray  # p.u., output in period 0
    base_mva: float
    rho: tuple  # (rho_pq, rho_va, rho_uc)
    name: str = ""

    def copy(self) -> "Grid":
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            kw[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        return Grid(**kw)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream)])))


def _topology(n: int, n_branch: int, rng: np.random.Generator):
    """Random spanning tree over points in the unit square, plus short chords."""
    pts = rng.random((n, 2))
    order = rng.permutation(n)
    frm, to = [], []
    placed = [int(order[0])]
    for k in range(1, n):
        b = int(order[k])
        P = np.asarray(placed)
        d = np.hypot(pts[P, 0] - pts[b, 0], pts[P, 1] - pts[b, 1])
        near = np.argsort(d, kind="stable")[: min(3, len(placed))]
        j = int(P[near[int(rng.integers(len(near)))]])
        frm.append(j)
        to.append(b)
        placed.append(b)
    n_chord = n_branch - (n - 1)
    if n_chord > 0:
        iu, ju = np.triu_indices(n, 1)
        key = set()
        for a, b in zip(frm, to):
            key.add((min(a, b), max(a, b)))
        mask = np.ones(iu.shape[0], dtype=bool)
        # drop pairs already joined by a tree edge
        tree_idx = np.array([a * n - a * (a + 1) // 2 + (b - a - 1) for (a, b) in key], dtype=np.int64)
        mask[tree_idx] = False
        iu, ju = iu[mask], ju[mask]
        d = np.hypot(pts[iu, 0] - pts[ju, 0], pts[iu, 1] - pts[ju, 1])
        w = np.exp(-d / 0.1)
        pick = rng.choice(iu.shape[0], size=n_chord, replace=False, p=w / w.sum())
        pick = np.sort(pick)
        frm.extend(int(x) for x in iu[pick])
        to.extend(int(x) for x in ju[pick])
    return np.asarray(frm, np.int32), np.asarray(to, np.int32)


def _load_shape(T: int) -> np.ndarray:
    h0 = 0 if T == 24 else 6
    h = (h0 + np.arange(T)) % 24
    return 1.0 + 0.3 * np.sin(2.0 * np.pi * (h - 9) / 24.0)


def make_grid(n_bus: int, n_branch: int, n_gen: int, T: int, seed: int = 0,
              load_seed: int | None = None, load_scale: float = 1.0,
              rho=(5e3, 1e4, 1e4), name: str = "", loading: float | None = None,
              q_ratio: float = 0.5, shunts: bool = False) -> Grid:
    """Draw one instance.

    `seed` fixes the network, generator fleet and base loads; `load_seed`, when
    given, multiplies every (t, bus) load by (1 + 0.05 N(0,1)) from its own
    stream (a load-profile scenario on the same network).  `shunts` adds, from
    a stream of its own (everything else is unchanged), bus shunts G^s, B^s
    (Eq. acopf balance equations) at about a third of the buses -- G^s ~
    U(0.005, 0.05), B^s ~ U(-0.1, 0.3) p.u., both nonzero, so that the bus
    projection's two balance multipliers are coupled -- and total line
    charging b ~ U(0.02, 0.3) p.u. (the pi model of Eq. acopf's flow
    equations) on about half of the lines.
    """
    if n_bus < 2 or n_branch < n_bus - 1 or n_gen < 1 or n_gen > n_bus or T < 1:
        raise ValueError("bad instance sizes")
    rg = _rng(seed, 1)
    frm, to = _topology(n_bus, n_branch, rg)
    rb = _rng(seed, 2)
    r = rb.uniform(0.005, 0.05, n_branch)
    x = rb.uniform(0.05, 0.3, n_branch)
    rate = rb.uniform(1.0, 3.0, n_branch)
    rl = _rng(seed, 3)
    base = rl.uniform(0.5, 1.5, n_bus)
    shape = _load_shape(T)
    loading = network_loading(n_bus) if loading is None else loading
    Pd = 0.7 * loading * load_scale * shape[:, None] * base[None, :]
    if load_seed is not None:
        rs = _rng(seed, 1000 + int(load_seed))
        Pd = Pd * (1.0 + 0.05 * rs.standard_normal((T, n_bus)))
    Qd = 0.33 * Pd
    rgn = _rng(seed, 4)
    gen_bus = np.sort(rgn.choice(n_bus, size=n_gen, replace=False)).astype(np.int32)
    raw = rgn.uniform(0.5, 1.5, n_gen)
    peak = float(Pd.sum(axis=1).max())
    Pmax = raw * (1.5 * peak / raw.sum())
    rc = _rng(seed, 5)
    c2 = rc.uniform(0.005, 0.05, n_gen)
    c1 = rc.uniform(10.0, 40.0, n_gen)
    c0 = rc.uniform(100.0, 500.0, n_gen)
    c_su = rc.uniform(200.0, 1000.0, n_gen)
    ref_bus = int(gen_bus[int(np.argmax(Pmax))])
    ones = np.ones(n_bus)
    Gs, Bs, br_b = np.zeros(n_bus), np.zeros(n_bus), np.zeros(n_branch)
    if shunts:
        rsh = _rng(seed, 6)
        on = rsh.random(n_bus) < 1.0 / 3.0
        on[int(rsh.integers(n_bus))] = True  # at least one shunt bus
        Gs = np.where(on, rsh.uniform(0.005, 0.05, n_bus), 0.0)
        Bs = np.where(on, rsh.uniform(-0.1, 0.3, n_bus), 0.0)
        Bs = np.where(on & (Bs == 0.0), 0.1, Bs)
        ch = rsh.random(n_branch) < 0.5
        ch[int(rsh.integers(n_branch))] = True
        br_b = np.where(ch, rsh.uniform(0.02, 0.3, n_branch), 0.0)
    return Grid(
        n_bus=n_bus, n_branch=n_branch, n_gen=n_gen, T=T, ref_bus=ref_bus,
        Pd=np.ascontiguousarray(Pd), Qd=np.ascontiguousarray(Qd),
        Gs=Gs, Bs=Bs, Vmin=0.9 * ones, Vmax=1.1 * ones,
        br_from=frm, br_to=to, br_r=r, br_x=x, br_b=br_b, br_rate=rate,
        gen_bus=gen_bus, Pmin=0.2 * Pmax, Pmax=Pmax, Qmin=-0.3 * Pmax, Qmax=q_ratio * Pmax,
        c2=c2, c1=c1, c0=c0, c_su=c_su, c_sd=np.zeros(n_gen),
        RU=0.5 * Pmax, RD=0.5 * Pmax, SU=0.5 * Pmax, SD=0.5 * Pmax,
        TU=np.full(n_gen, 2, np.int32), TD=np.full(n_gen, 2, np.int32),
        u0=np.ones(n_gen, np.int32), L0=np.zeros(n_gen, np.int32), F0=np.zeros(n_gen, np.int32),
        p0=0.5 * Pmax, base_mva=100.0, rho=tuple(float(v) for v in rho), name=name,
    )


# Workload descriptions (sizes of the paper-shaped synthetic configs).
CONFIGS = {
    "c1_9bus_T6": "9-bus, 9 branches, 3 generators, T=6, seed 0 (case9 penalties)",
    "c2_118bus_T24x3": "118-bus, 186 branches, 54 generators, T=24, load-profile seeds 0..2 (case118 penalties)",
    "c4_batch64": "64 uneven instances: buses U{30..500}, branches round(1.5 n), generators round(0.3 n), "
                  "T in {12,18,24}, load scale U(0.8,1.1) (case300 penalties)",
    "c5_2000bus_T24x16": "2000-bus, 3200 branches, 500 generators, T=24, 16 load scenarios (case300 penalties)",
}


def config_instances(name: str, n_instances: int | None = None, shunts: bool = False) -> List[Grid]:
    """Instances of a named workload; `n_instances` truncates batched ones;
    `shunts` adds bus shunts and line charging (see make_grid) to each."""
    if name == "c1_9bus_T6":
        out = [make_grid(9, 9, 3, 6, seed=0, rho=RHO_TABLE["case9"], name=name, shunts=shunts)]
    elif name == "c2_118bus_T24x3":
        out = [make_grid(118, 186, 54, 24, seed=0, load_seed=s, rho=RHO_TABLE["case118"],
                         name=f"{name}[{s}]", shunts=shunts) for s in range(3)]
    elif name == "c4_batch64":
        r = _rng(0, 77)
        out = []
        for k in range(64):
            n = int(r.integers(30, 501))
            T = int(r.choice([12, 18, 24]))
            sc = float(r.uniform(0.8, 1.1))
            out.append(make_grid(n, int(round(1.5 * n)), max(1, int(round(0.3 * n))), T, seed=100 + k,
                                 load_scale=sc, rho=RHO_TABLE["case300"], name=f"{name}[{k}]", shunts=shunts))
    elif name == "c5_2000bus_T24x16":
        out = [make_grid(2000, 3200, 500, 24, seed=0, load_seed=s, rho=RHO_TABLE["case300"],
                         name=f"{name}[{s}]", shunts=shunts) for s in range(16 if n_instances is None else n_instances)]
    else:
        raise KeyError(name)
    if n_instances is not None:
        out = out[:n_instances]
    return out


def stack_sizes(grids: Sequence[Grid]) -> dict:
    """Per-sweep work counts of a batch (items, not arithmetic)."""
    bp = sum(g.T * g.n_branch for g in grids)
    gp = sum(g.T * g.n_gen for g in grids)
    up = sum(g.T * g.n_bus for g in grids)
    return {"branch_periods": bp, "gen_periods": gp, "bus_periods": up,
            "dps": sum(g.n_gen for g in grids)}
