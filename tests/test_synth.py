"""The seeded input generator: reproducible, connected, sized as configured."""
import numpy as np

from paper_2310_13145_b300 import synth


def _connected(g):
    par = list(range(g.n_bus))

    def f(a):
        while par[a] != a:
            a = par[a]
        return a
    for a, b in zip(g.br_from, g.br_to):
        par[f(a)] = f(b)
    return len({f(i) for i in range(g.n_bus)}) == 1


def test_configs_have_the_stated_sizes():
    g1 = synth.config_instances("c1_9bus_T6")
    assert (g1[0].n_bus, g1[0].n_branch, g1[0].n_gen, g1[0].T) == (9, 9, 3, 6)
    g2 = synth.config_instances("c2_118bus_T24x3")
    assert len(g2) == 3 and all((g.n_bus, g.n_branch, g.n_gen, g.T) == (118, 186, 54, 24) for g in g2)
    # same network, different load profiles
    assert np.array_equal(g2[0].br_from, g2[1].br_from) and not np.array_equal(g2[0].Pd, g2[1].Pd)
    for g in g1 + g2:
        assert _connected(g)
        assert len(set(zip(np.minimum(g.br_from, g.br_to), np.maximum(g.br_from, g.br_to)))) == g.n_branch
        assert abs(g.Pmax.sum() - 1.5 * g.Pd.sum(axis=1).max()) < 1e-9 * g.Pmax.sum()


def test_reproducible():
    a = synth.make_grid(50, 75, 15, 12, seed=3, load_seed=1)
    b = synth.make_grid(50, 75, 15, 12, seed=3, load_seed=1)
    for k, v in vars(a).items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, getattr(b, k)), k
