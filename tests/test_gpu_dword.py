"""The device's double-word arithmetic (the FP32-pair operations of the bus
kernel's row updates) gives the same bits as the same header built for the
host, whose error bounds test_dword.py checks against exact arithmetic: the
device neither contracts, reorders nor flushes any of its steps."""
import numpy as np
import pytest

from tests import test_dword as H

pytestmark = pytest.mark.gpu


def _inputs():
    n = 4000
    x, y, z = H.sample(n, 31, -20, 20), H.sample(n, 32, -20, 20), H.sample(n, 33, -20, 20)
    y[: n // 4] = -x[: n // 4] * (1.0 + np.random.default_rng(34).normal(0, 1e-9, n // 4))
    z[: n // 4] = -(x[: n // 4] * y[: n // 4]) * (1.0 + np.random.default_rng(35).normal(0, 1e-9, n // 4))
    sp = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 2.0 ** -100, 1e-200, 1e200, np.inf, np.nan, np.pi])
    return (np.concatenate([x, sp]), np.concatenate([y, sp[::-1]]), np.concatenate([z, sp]))


@pytest.mark.parametrize("op", range(8))
def test_device_ops_match_host_bits(ucac_mod, tmp_path, op):
    host = H.build_host(tmp_path)
    x, y, z = _inputs()
    ref = H.run_ops(host, op, x, y, z)
    got = ucac_mod.ucac_probe_dw(op, x, y, z)
    same = (ref.view(np.uint64) == got.view(np.uint64)) | (np.isnan(ref) & np.isnan(got))
    assert same.all(), (op, np.argwhere(~same)[:5], ref[~same.all(axis=1)][:3], got[~same.all(axis=1)][:3])


def test_probe_dw_arguments(ucac_mod):
    with pytest.raises(ucac_mod.UcacError):
        ucac_mod.ucac_probe_dw(8, np.zeros(3))
    assert ucac_mod.ucac_probe_dw(1, np.zeros(0)).shape == (0, 4)
