"""Pins of the oracle's ground extraction (§III-A, Eq. 1 in its tangent form)."""
import math

import numpy as np
import pytest

import oracle

H = 1.7  # sensor height above the ground plane (m)


def _plane_ranges(elev, slopes, h=H):
    """Ranges (double) of beams at elevations elev hitting the lines z = -h + x tan(phi),
    one column per slope phi; 0 where a beam misses (or hits beyond 200 m)."""
    R, C = len(elev), len(slopes)
    out = np.zeros((R, C))
    for r, e in enumerate(elev):
        for c, phi in enumerate(slopes):
            den = math.cos(e) * math.tan(phi) - math.sin(e)
            if den > 1e-9:
                t = h / den
                if t < 200.0:
                    out[r, c] = t
    return out


def _beta(d1, e1, d2, e2):
    """Angle at the upper point A between the ray back to the sensor and the segment to
    the lower point B, from coordinates (double): independent of Eq. 1."""
    ax, az = d1 * math.cos(e1), d1 * math.sin(e1)
    bx, bz = d2 * math.cos(e2), d2 * math.sin(e2)
    ux, uz = -ax, -az
    vx, vz = bx - ax, bz - az
    return math.atan2(abs(ux * vz - uz * vx), ux * vx + uz * vz)


def test_hand_case():
    """Beams at 0 and -90 degrees, both readings 1: the segment between the points is the
    diagonal, beta = 45 degrees, gamma = 0, so ground iff theta reaches 45 degrees; the
    first row takes the second row's decision."""
    e = np.radians([0.0, -90.0])
    r = np.array([[1.0], [1.0]], np.float32)
    assert oracle.ground(r, e, math.radians(50)).ravel().tolist() == [True, True]
    assert oracle.ground(r, e, math.radians(40)).ravel().tolist() == [False, False]
    r2 = np.array([[1.0], [0.0]], np.float32)  # no reading below: nothing to compare
    assert not oracle.ground(r2, e, math.radians(50)).any()


@pytest.mark.parametrize("theta_deg", [10.0, 2.0, 0.1])
def test_flat_ground_is_ground(theta_deg):
    elev = np.radians(np.linspace(-2.0, -24.8, 64))
    rng = _plane_ranges(elev, [0.0] * 8).astype(np.float32)
    g = oracle.ground(rng, elev, math.radians(theta_deg))
    assert (rng > 0).all() and g.all()


def test_wall_is_not_ground():
    elev = np.radians(np.linspace(15.0, -24.8, 64))
    rng = np.array([[5.0 / math.cos(e)] * 4 for e in elev], np.float32)  # wall at x = 5
    assert not oracle.ground(rng, elev, math.radians(10)).any()


@pytest.mark.parametrize("theta_deg", [10.0, 4.0])
def test_slopes_against_geometry(theta_deg):
    """Inclined planes of slope phi: every reading's decision equals |beta - gamma| <=
    theta with beta taken from the points' coordinates in double (readings rounded to
    fp32 first), except within 1e-4 rad of the bound."""
    theta = math.radians(theta_deg)
    elev = np.radians(np.linspace(-3.0, -24.8, 48))
    slopes = np.radians([-25, -15, -12, -9.9, -8, -3.9, 0, 2, 3.95, 5, 9.5, 11, 14, 20])
    rng = _plane_ranges(elev, slopes).astype(np.float32)
    g = oracle.ground(rng, elev, theta)
    checked = 0
    for c in range(len(slopes)):
        for r in range(1, len(elev)):
            d1, d2 = float(rng[r - 1, c]), float(rng[r, c])
            if d1 <= 0 or d2 <= 0:
                assert not g[r, c]
                continue
            beta = _beta(d1, float(elev[r - 1]), d2, float(elev[r]))
            off = abs(beta - (-float(elev[r - 1])))
            if abs(off - theta) < 1e-4:
                continue
            assert g[r, c] == (off <= theta), (r, c, math.degrees(beta))
            checked += 1
        # the first row decides as the second
        assert g[0, c] == (g[1, c] and rng[0, c] > 0)
    assert checked > 400


def test_height_exception_keeps_raised_surfaces():
    """A flat roof 1.5 m above the ground plane is horizontal but lies above the line from
    the wheels rising at theta, so it is kept; the ground plane is removed."""
    elev = np.radians(np.linspace(-2.0, -24.8, 64))
    theta = math.radians(10)
    ground = _plane_ranges(elev, [0.0] * 3).astype(np.float32)
    roof = _plane_ranges(elev, [0.0] * 3, h=0.2).astype(np.float32)
    rng = np.concatenate([ground, roof], axis=1)
    no_exc = oracle.ground(rng, elev, theta)
    exc = oracle.ground(rng, elev, theta, mount_height=H)
    assert no_exc.all()
    assert exc[:, :3].all() and not exc[:, 3:].any()


def test_disabled_and_label_composition():
    g = np.random.default_rng(5)
    elev = np.radians(np.linspace(5.0, -20.0, 12))
    rng = g.uniform(2.0, 8.0, (12, 40)).astype(np.float32)
    assert not oracle.ground(rng, elev, 0.0).any()
    mask = oracle.ground(rng, elev, math.radians(30))
    a = oracle.label_ground(rng, elev, 2 * math.pi / 40, 0.5, 2, True, math.radians(30))
    b = oracle.label(np.where(mask, 0, rng).astype(np.float32), elev, 2 * math.pi / 40, 0.5, 2, True)
    assert np.array_equal(a, b)
    assert (a.reshape(12, 40)[mask] == -1).all()


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_synthetic_ground_truth(name):
    """On the ray-cast scenes, the readings removed are nearly all hits of the ground plane
    (object id 0) and most ground hits are removed: the ones kept lack a usable reading
    above (dropout, an object in front) or sit in noise."""
    from paper_2003_00575_gb300 import synth
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[name]()
    g = oracle.ground(f.range, f.sensor.elevation, math.radians(10), 1.7)
    truth = (f.object_id == 0) & (f.range > 0)
    precision = (g & truth).sum() / max(g.sum(), 1)
    recall = (g & truth).sum() / max(truth.sum(), 1)
    assert precision > 0.95 and recall > 0.6, (precision, recall)
