"""The OpenMP build of the oracle (x-step subproblems of every generator and
line on several host threads) gives the same bits as the plain build: the
subproblems are independent and every sum stays sequential."""
import numpy as np

import oracle
from paper_2310_13145_b300 import synth


def test_openmp_build_is_bit_identical():
    g = synth.config_instances("c2_118bus_T24x3", 1)[0]
    a = oracle.Oracle(g)
    assert oracle.threads(4) == 4
    b = oracle.Oracle(g, omp=True)
    for _ in range(6):
        a.sweep()
        b.sweep()
        assert np.array_equal(a.state_vector(), b.state_vector())
    ra, rb = a.residuals(), b.residuals()
    assert ra == rb
