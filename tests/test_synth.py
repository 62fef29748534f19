"""The seeded heterogeneous Ks field has the stated log-normal statistics and separable exponential correlation."""
import math

import numpy as np

from paper_2112_05051_gb300 import synth


def test_ks_field_statistics():
    grid = synth.Grid(64, 64, 64)
    sigma = 1.5
    ks = synth.ks_field(grid, 3, sigma, (4.0, 4.0, 2.0))
    g = (np.log10(ks) - math.log10(9.44e-3)) / sigma
    assert abs(g.mean()) < 0.15 and abs(g.std() - 1.0) < 0.15
    g3 = g.reshape(grid.shape)
    for ax, ell in ((2, 4.0), (1, 4.0), (0, 2.0)):
        a = np.moveaxis(g3, ax, 0)
        r = np.mean(a[1:] * a[:-1]) / np.mean(a * a)
        assert abs(r - math.exp(-1.0 / ell)) < 0.05
    # deterministic in the seed
    np.testing.assert_array_equal(ks, synth.ks_field(grid, 3, sigma, (4.0, 4.0, 2.0)))


def test_dt_ramp_schedule():
    d = synth.dt_schedule("ramp1to30", 20)
    assert d[0] == 1.0 and d[-1] == 30.0 and len(d) == 20
    assert all(b > a for a, b in zip(d, d[1:]))
