"""The C ABI library loads and exports every entry point declared in
include/ucac.h; host-side argument and grid validation (which runs before any
CUDA call) returns the documented error codes.  No GPU needed."""
import os
import re

import numpy as np
import pytest

from paper_2310_13145_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    hdr = open(os.path.join(ROOT, "include", "ucac.h")).read()
    return set(re.findall(r"^\s*(?:[A-Za-z_][\w \*]*?)\b(ucac_\w+)\s*\(", hdr, re.M))


def test_every_declared_symbol_is_exported(ucac_mod):
    L = ucac_mod.lib()
    decl = declared()
    assert decl == set(ucac_mod.EXPORTS)
    for s in decl:
        assert hasattr(L, s), s


def test_oracle_and_library_share_nothing():
    # the oracle never loads the CUDA library and vice versa
    src = open(os.path.join(ROOT, "oracle", "ucac_oracle.c")).read() + open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2310_13145_b300" not in src and "ucac.h" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2310_13145_b300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2310_13145_b300", "csrc", f)).read().lower()
    for f in ("ucac.py", "synth.py", "build.py"):
        txt = open(os.path.join(ROOT, "paper_2310_13145_b300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt


def _bad(g, **kw):
    g = g.copy()
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("mut,code", [
    (dict(br_from=np.array([0, 0, 0, 0, 0, 0, 0, 0, 0], np.int32), br_to=np.array([1, 1, 1, 1, 1, 1, 1, 1, 1], np.int32)), -2),  # disconnected
    (dict(br_r=np.zeros(9), br_x=np.zeros(9)), -2),
    (dict(Vmin=np.full(9, 1.2)), -2),
    (dict(ref_bus=99), -2),
    (dict(u0=np.full(3, 2, np.int32)), -2),
])
def test_invalid_grids_rejected_before_any_device_work(ucac_mod, mut, code):
    g = synth.config_instances("c1_9bus_T6")[0]
    with pytest.raises(ucac_mod.UcacError) as e:
        ucac_mod.ucac_create(_bad(g, **mut))
    assert f"error {code}" in str(e.value)
    assert ucac_mod.ucac_last_error(None)


def test_nan_load_rejected(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    Pd = g.Pd.copy()
    Pd[2, 3] = np.nan
    with pytest.raises(ucac_mod.UcacError, match="error -2"):
        ucac_mod.ucac_create(_bad(g, Pd=Pd))


def test_bad_horizon_and_params(ucac_mod):
    g = synth.config_instances("c1_9bus_T6")[0]
    with pytest.raises(ucac_mod.UcacError, match="error -2"):
        ucac_mod.ucac_create(g, horizon=g.T + 1)
    with pytest.raises(ucac_mod.UcacError, match="error -1"):
        ucac_mod.ucac_create(g, params=ucac_mod.ucac_default_params(K_N=0))


def test_noalloc_size_limit_is_host_side(ucac_mod):
    with pytest.raises(ucac_mod.UcacError, match="static limit"):
        ucac_mod.ucac_ucdp_noalloc(20000, 168, 1e4, *([1] * 12))
