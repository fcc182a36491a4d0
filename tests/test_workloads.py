"""The synthetic input recipe: the generators produce the fields the
workloads are defined by (CPU only).

* Gaussian random fields: seeded white noise smoothed by a Gaussian of
  sigma cells, zero mean, exact target standard deviation.  Smoothing white
  noise with a Gaussian of width sigma gives the correlation
  exp(-d^2 / (4 sigma^2)) at lag d, which the field must show.
* Channel fields: background k = 1 and axis-aligned rectangles at k = 1e6,
  so log k takes exactly two values.
* Regular block partitions and the TPFA matrices are pinned in
  test_oracle_pins.py.
"""

import numpy as np
import pytest

from workloads.darcy import channel_field, grf_logk


def _lag_corr(x, d, axis):
    a = np.moveaxis(x, axis, 0)
    return float(np.corrcoef(a[:-d].ravel(), a[d:].ravel())[0, 1])


@pytest.mark.parametrize("sigma", [2.0, 4.0])
def test_grf_moments_and_correlation_length(sigma):
    x = grf_logk((256, 256), sigma, 2.0, 7)
    assert abs(x.mean()) < 1e-12
    assert abs(x.std() - 2.0) < 1e-12
    for d in (1, 2):
        for axis in (0, 1):
            assert abs(_lag_corr(x, d, axis) - np.exp(-d * d / (4 * sigma * sigma))) < 0.025


def test_grf_three_dimensional_and_seeded():
    x = grf_logk((48, 48, 48), 3.0, 1.0, 1)
    assert x.shape == (48, 48, 48) and x.flags.c_contiguous
    assert abs(x.mean()) < 1e-12 and abs(x.std() - 1.0) < 1e-12
    for axis in range(3):
        assert abs(_lag_corr(x, 2, axis) - np.exp(-4 / 36)) < 0.025
    assert np.array_equal(x, grf_logk((48, 48, 48), 3.0, 1.0, 1))
    assert not np.array_equal(x, grf_logk((48, 48, 48), 3.0, 1.0, 2))


def test_channel_field_two_values_and_coverage():
    logk = channel_field((1024, 1024))
    vals = np.unique(logk)
    assert np.array_equal(vals, [0.0, np.log(1e6)])
    # 200 channels of mean width 3 and mean length 288 cover at most about
    # 16 % of the grid; overlaps and clipping at the domain leave less
    frac = float((logk > 0).mean())
    assert 0.08 < frac < 0.17
    assert np.array_equal(logk, channel_field((1024, 1024)))
    assert not np.array_equal(logk, channel_field((1024, 1024), seed=1))


def test_channel_field_rectangles_are_axis_aligned_and_sized():
    """One channel at a time: a single rectangle of width 2..4 and length
    64..512 along x or y, clipped only at the far edges of the domain."""
    for seed in range(20):
        logk = channel_field((600, 600), nchannels=1, seed=seed)
        ys, xs = np.nonzero(logk > 0)
        h, w = ys.max() - ys.min() + 1, xs.max() - xs.min() + 1
        assert len(ys) == h * w                      # a full rectangle
        short, long_ = sorted((h, w))
        assert 1 <= short <= 4 and long_ <= 512
        if ys.max() < 599 and xs.max() < 599:        # not clipped
            assert 2 <= short <= 4 and 64 <= long_ <= 512


def test_batch_of_uneven_systems_recipe():
    """The batch generator's draws, on small side ranges: 24 2-D and 24 3-D
    systems, sides, log-std and m inside their ranges, 8 N(0,1) right-hand
    sides each, 8^d blocks with partial blocks at the far edges."""
    from workloads.darcy import make_batch48_uneven
    ws = make_batch48_uneven(lo2=16, hi2=24, lo3=8, hi3=12)
    assert len(ws) == 48
    for i, w in enumerate(ws):
        d = 3 if i >= 24 else 2
        side = w.shape[0]
        assert len(w.shape) == d and all(s == side for s in w.shape)
        assert (8 <= side <= 12) if d == 3 else (16 <= side <= 24)
        assert 2.0 - 1e-12 <= w.logk.std() <= 3.0 + 1e-12
        assert 4 <= w.m <= 8 and w.nrhs == 8
        assert w.nparts == ((side + 7) // 8) ** d
        assert abs(w.rhs.mean()) < 0.2 and 0.8 < w.rhs.std() < 1.2
    assert len({w.shape[0] for w in ws}) > 4          # uneven sizes
    assert len({w.m for w in ws}) > 1
