"""Pins of the oracle's exact-ray horizontal constants (§III-B / §III-B-2: the angle
between two measurements, adjusted to the offset): K = 2 - 2 cos(alpha) with alpha the
true angle between the rays of one row k columns apart."""
import math

import numpy as np
import pytest

import oracle


def test_horizon_row_equals_the_paper_table():
    """At elevation 0 the true angle is k times the step: the two tables agree exactly."""
    elev = np.array([0.0, 0.0, 0.0])
    step = 2 * math.pi / 1800
    assert np.array_equal(oracle.tables(elev, step, 5, True)[1], oracle.tables(elev, step, 5)[1])


def test_against_the_dot_product():
    """K from the dot product of the two unit rays (double), cos(alpha) = cos^2 e cos(k step)
    + sin^2 e: the table is that value rounded to fp32 (within one ulp of it)."""
    g = np.random.default_rng(3)
    elev = np.radians(g.uniform(-40, 40, 64))
    step = 2 * math.pi / 2048
    kv, kh = oracle.tables(elev, step, 8, True)
    for r, e in enumerate(elev):
        for k in range(1, 9):
            u = np.array([math.cos(e), 0.0, math.sin(e)])
            v = np.array([math.cos(e) * math.cos(k * step), math.cos(e) * math.sin(k * step),
                          math.sin(e)])
            K = float(np.sum((u - v) ** 2))  # |u - v|^2 = 2 - 2 cos(alpha), no cancellation
            got = float(kh[r, k - 1])
            assert abs(got - K) <= 2 * np.spacing(np.float32(K)), (r, k, got, K)
    # the vertical table does not change
    assert np.array_equal(kv, oracle.tables(elev, step, 8)[0])


def test_predicate_matches_point_distances():
    """With the exact constants Eq. 2 is the 3D distance between the two points: decide it
    from the points' coordinates in double and compare, away from the threshold."""
    g = np.random.default_rng(4)
    elev = np.radians(np.linspace(25, -25, 9))
    C = 360
    step = 2 * math.pi / C
    delta = 0.3
    kh = oracle.tables(elev, step, 4, True)[1]
    n = 0
    for _ in range(4000):
        r = int(g.integers(0, 9))
        k = int(g.integers(1, 5))
        a = float(np.float32(g.uniform(2, 30)))
        b = float(np.float32(a + g.uniform(-0.4, 0.4)))
        e = elev[r]
        pa = a * np.array([math.cos(e), 0.0, math.sin(e)])
        pb = b * np.array([math.cos(e) * math.cos(k * step), math.cos(e) * math.sin(k * step),
                           math.sin(e)])
        d = float(np.linalg.norm(pa - pb))
        if abs(d - delta) < 1e-4:
            continue
        assert oracle.pred(a, b, float(kh[r, k - 1]), delta) == (d <= delta), (r, k, a, b, d)
        n += 1
    assert n > 3000


def test_labels_differ_only_through_the_table():
    """Rows far from the horizon join fewer horizontal neighbours with the paper's (larger)
    constant than with the exact one; at the horizon nothing changes."""
    g = np.random.default_rng(8)
    elev = np.radians(np.linspace(30, -30, 21))
    rng = np.full((21, 200), 10.0, np.float32) + g.normal(0, 0.01, (21, 200)).astype(np.float32)
    step = 2 * math.pi / 200
    e_paper = oracle.edges(rng, elev, step, 0.3, 1, True)
    e_exact = oracle.edges(rng, elev, step, 0.3, 1, True, exact_ray=True)
    h = 1  # horizontal offset-1 bit
    assert ((e_exact & h) >= (e_paper & h)).all()  # a smaller K never removes an edge
    assert (e_exact[10] == e_paper[10]).all()      # the horizon row
    assert (e_exact & h).sum() > (e_paper & h).sum()
