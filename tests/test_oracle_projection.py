"""Pins of the oracle's spherical projection and scatter (§I, Fig. 1; §IV-B on the
one-to-one matching of points and range-image cells).  No GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_00575_gb300 import synth


def _double_assignment(xyz, sensor):
    """Pixel by double-precision angles (atan2) against double boundaries, plus the angular
    distance to the nearest boundary, for comparison with the oracle's fp32 sign tests."""
    x, y, z = (xyz[:, i].astype(np.float64) for i in range(3))
    rho = np.hypot(x, y)
    phi = np.mod(np.arctan2(y, x), 2 * math.pi)
    theta = np.arctan2(z, rho)
    C = sensor.cols
    col = np.floor(phi / sensor.az_step).astype(np.int64) % C
    dcol = np.abs(phi / sensor.az_step - np.round(phi / sensor.az_step)) * sensor.az_step
    order = np.argsort(sensor.elevation)
    es = sensor.elevation[order]
    bounds = np.r_[es[0] - (es[1] - es[0]) / 2, (es[:-1] + es[1:]) / 2,
                   es[-1] + (es[-1] - es[-2]) / 2]
    j = np.searchsorted(bounds, theta, side="right") - 1
    inside = (j >= 0) & (j < len(es))
    jj = np.clip(j, 0, len(es) - 1)
    drow = np.min(np.abs(theta[:, None] - bounds[None, :]), axis=1)
    pix = np.where(inside, order[jj] * C + col, -1)
    return pix, np.minimum(dcol, drow)


def test_round_trip_pixel_centres():
    f = synth.config_c2()
    s = f.sensor
    g = np.random.default_rng(5)
    xyz = synth.pixel_cloud(g, s, f.range, jitter=0.0)
    rimg, pix, win = oracle.project(xyz, s.rows, s.cols, s.elevation, s.az_step)
    valid = (f.range > 0).reshape(-1)
    idx = np.arange(s.rows * s.cols)
    assert np.array_equal(pix[valid], idx[valid])
    assert np.all(pix[~valid] == -1)
    # recomputed range within 2 ulp of the original
    a = rimg.reshape(-1)[valid].astype(np.float64)
    b = f.range.reshape(-1)[valid].astype(np.float64)
    ulp = np.spacing(f.range.reshape(-1)[valid]).astype(np.float64)
    assert np.all(np.abs(a - b) <= 2 * ulp)
    assert np.array_equal(win[valid], idx[valid])


def test_round_trip_with_quarter_bin_jitter():
    f = synth.config_c3()
    s = f.sensor
    rimg, pix, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
    valid = (f.range > 0).reshape(-1)
    idx = np.arange(s.rows * s.cols)
    assert np.array_equal(pix[valid], idx[valid])
    assert np.all(pix[~valid] == -1)


def test_agrees_with_double_angles_away_from_boundaries():
    s = synth.make_sensor(32, 1024, -20.0, 20.0)
    g = np.random.default_rng(9)
    n = 200_000
    d = g.uniform(0.5, 100, n)
    az = g.uniform(0, 2 * math.pi, n)
    el = g.uniform(math.radians(-24), math.radians(24), n)
    xyz = np.stack([d * np.cos(el) * np.cos(az), d * np.cos(el) * np.sin(az), d * np.sin(el)],
                   1).astype(np.float32)
    _, pix, _ = oracle.project(xyz, s.rows, s.cols, s.elevation, s.az_step)
    want, dist = _double_assignment(xyz, s)
    far = dist > 1e-6
    assert far.mean() > 0.99
    assert np.array_equal(pix[far], want[far])
    assert np.any(want == -1) and np.any(pix == -1)


def test_conflicts_nearest_then_lowest_index():
    s = synth.make_sensor(16, 1800, -15.0, 15.0)
    r, c = 7, 100
    e = s.elevation[r]
    a = (c + 0.5) * s.az_step
    u = np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a), math.sin(e)])
    pts = np.stack([u * 10.0, u * 5.0, u * 5.0, u * 8.0]).astype(np.float32)
    rimg, pix, win = oracle.project(pts, s.rows, s.cols, s.elevation, s.az_step)
    p = r * s.cols + c
    assert np.all(pix == p)
    assert win[p] == 1  # ranges 10, 5, 5, 8: nearest is 5, tie goes to index 1
    assert rimg.reshape(-1)[p] == np.float32(np.linalg.norm(pts[1].astype(np.float32)))
    assert np.count_nonzero(rimg) == 1


def test_invalid_points_dropped():
    s = synth.make_sensor(16, 1800, -15.0, 15.0)
    pts = np.array([[0, 0, 0], [np.nan, 1, 0], [np.inf, 0, 0], [0, 0, 5.0],
                    [10.0, 0.0, 10.0]], np.float32)  # origin, NaN, inf, on-axis, 45 deg up
    _, pix, _ = oracle.project(pts, s.rows, s.cols, s.elevation, s.az_step)
    assert np.all(pix == -1)


def test_scatter():
    labels = np.array([[5, -1], [2, 3]], np.int32)
    pix = np.array([0, 1, 2, 3, -1, 0], np.int32)
    np.testing.assert_array_equal(oracle.scatter(labels, pix), [5, -1, 2, 3, -1, 5])


@pytest.mark.parametrize("rows", [1])
def test_projection_needs_two_rows(rows):
    with pytest.raises(ValueError):
        oracle.proj_tables(rows, 8, np.array([0.0]), 2 * math.pi / 8)
