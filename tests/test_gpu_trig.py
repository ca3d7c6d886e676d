"""The polar line kernel's cos/sin (table of cos(k/256), sin(k/256) rotated
by the Taylor series of the remainder) against numpy's cos/sin on the
device."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PI_BOUND = 3.14159265358979  # the angle bound of the polar line variables
TRIG_N = 256  # table resolution


def _angles():
    rng = np.random.default_rng(7)
    k = np.arange(-804, 805)
    pts = [np.array([0.0, -0.0, 1e-300, -1e-300, 1e-9, -1e-9, PI_BOUND, -PI_BOUND, np.pi / 2, -np.pi / 2]),
           k / TRIG_N,                                      # table points (remainder 0)
           (k[:-1] + 0.5) / TRIG_N,                         # halfway: rint ties
           np.nextafter((k[:-1] + 0.5) / TRIG_N, np.inf),   # just past the ties
           rng.uniform(-PI_BOUND, PI_BOUND, 20000),
           rng.normal(0.0, 0.1, 20000).clip(-PI_BOUND, PI_BOUND)]  # line angles are mostly small
    return np.concatenate(pts)


def test_cossin_against_numpy(ucac_mod):
    d = _angles()
    c, s = ucac_mod.ucac_probe_cossin(d)
    err_c = np.abs(c - np.cos(d))
    err_s = np.abs(s - np.sin(d))
    # absolute error within a few units in the last place of 1
    assert err_c.max() <= 1e-15, (err_c.max(), d[np.argmax(err_c)])
    assert err_s.max() <= 1e-15, (err_s.max(), d[np.argmax(err_s)])
    # tiny angles keep their relative accuracy (sin d = d to the last place)
    small = np.abs(d) < 1e-8
    assert np.all(np.abs(s[small] - d[small]) <= 2.3e-16 * np.abs(d[small]))
    assert np.all(c[small] == 1.0)
    # cos^2 + sin^2 = 1
    assert np.max(np.abs(c * c + s * s - 1.0)) <= 2e-15


def test_cossin_empty(ucac_mod):
    c, s = ucac_mod.ucac_probe_cossin(np.zeros(0))
    assert c.size == 0 and s.size == 0
