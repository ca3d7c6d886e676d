"""Writes tests/golden/uc_dp_cases.json: fixed UC subproblems and their optimal
cost and schedule, found by the brute-force enumerator in oracle/bruteforce.py
(every schedule, Eq. set:UC checked as written).  Calls nothing but oracle/."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import bruteforce as bf  # noqa: E402


def main():
    rng = np.random.Generator(np.random.Philox(12345))
    out = []
    for n in range(12):
        T = int(rng.integers(3, 10))
        TU = int(rng.integers(1, min(T, 4) + 1))
        TD = int(rng.integers(1, min(T, 4) + 1))
        u0 = int(rng.integers(0, 2))
        K0 = int(rng.integers(0, 2))
        L, F = (K0, 0) if u0 else (0, K0)
        c = dict(name=f"case{n}", T=T, TU=TU, TD=TD, u0=u0, K0=K0, L=L, F=F,
                 c0=float(rng.uniform(0, 400)), csu=float(rng.uniform(0, 900)), csd=float(rng.uniform(0, 300)),
                 rho=1e3)
        ubar = rng.uniform(0, 1, (3, T))
        y = rng.normal(0, 300, (3, T))
        z = rng.normal(0, 0.05, (3, T))
        best, u = bf.best_schedule(T, u0, L, F, TU, TD, c["c0"], c["csu"], c["csd"], c["rho"], ubar, y, z)
        c.update(ubar=ubar.tolist(), y=y.tolist(), z=z.tolist(), best=best, schedule=[int(v) for v in u])
        out.append(c)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "uc_dp_cases.json")
    json.dump(out, open(path, "w"), indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
