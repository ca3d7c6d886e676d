"""The autotuner and the block sizes it chooses: any block size gives the
same iterate bit for bit (work is split in warp-sized granules of one
instance each); a cache entry is applied without timing."""
import numpy as np
import pytest

from paper_2310_13145_b300 import synth

pytestmark = pytest.mark.gpu


def _key(ucac_mod, grids, line_form=1):
    import torch
    ngp = sum(g.T * g.n_gen for g in grids)
    nbp = sum(g.T * g.n_branch for g in grids)
    nup = sum(g.T * g.n_bus for g in grids)
    return f"{torch.cuda.get_device_name(0)}|{len(grids)}|{ngp}|{nbp}|{nup}|{line_form}"


@pytest.mark.parametrize("sizes", [(32, 32, 32, 32, 32), (256, 256, 128, 256, 256), (64, 128, 32, 256, 64)])
def test_block_sizes_change_no_result(ucac_mod, tmp_path, sizes):
    grids = synth.config_instances("c2_118bus_T24x3") + [synth.make_grid(13, 16, 4, 7, seed=3)]
    ref = ucac_mod.Handle(grids)
    ref.enqueue(6)
    cache = tmp_path / "tune.txt"
    cache.write_text(_key(ucac_mod, grids) + " " + " ".join(str(v) for v in sizes) + "\n")
    h = ucac_mod.Handle(grids)
    got = h.autotune(2, str(cache))
    assert tuple(got.values()) == sizes  # cache hit applied as written
    h.enqueue(6)
    for k in range(len(grids)):
        assert np.array_equal(h.export(k), ref.export(k)), k
    h.close()
    ref.close()


def test_autotune_times_and_caches(ucac_mod, tmp_path):
    grids = synth.config_instances("c2_118bus_T24x3")
    cache = tmp_path / "tune.txt"
    h = ucac_mod.Handle(grids)
    h.enqueue(3)
    before = h.export(0)
    t1 = h.autotune(2, str(cache))
    assert np.array_equal(h.export(0), before)  # iterate restored
    assert all(v in (32, 64, 128, 256) for v in t1.values())
    assert cache.read_text().count("\n") == 1
    h2 = ucac_mod.Handle(grids)
    assert h2.autotune(2, str(cache)) == t1
    assert cache.read_text().count("\n") == 1
    h.close()
    h2.close()
