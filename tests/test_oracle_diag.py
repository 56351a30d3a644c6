"""Pins of the oracle's diagonal Map Connections (§III-B-2, "MCs along the main diagonal"):
pixel (r, c) also joined to (r+k, c+k) and (r+k, c-k), k = 1..S, with Eq. 3's constant
from the true angle between the two beams' rays.  Checked against a hand-worked frame,
the dot-product definition of the constant and 3D point distances, all-pairs brute force
on tiny grids, an independently built edge list through scipy's connected components, and
the nesting of the partitions with and without the diagonals."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "diag_hand_3x4.json")


def _rays(elev, az_step, r, k):
    e1, e2, ph = elev[r], elev[r + k], k * az_step
    u1 = np.array([math.cos(e1), 0.0, math.sin(e1)])
    u2 = np.array([math.cos(e2) * math.cos(ph), math.cos(e2) * math.sin(ph), math.sin(e2)])
    return u1, u2


def test_hand_frame():
    g = json.load(open(GOLDEN))
    elev = np.radians(g["elevation_deg"])
    az = math.radians(g["az_step_deg"])
    rng = np.array(g["range"], np.float32)
    np.testing.assert_array_equal(oracle.tables_diag(elev, az, 2), np.array(g["kd"], np.float32))
    for case in g["cases"]:
        got = oracle.label(rng, elev, az, case["delta"], case["skip"], wrap=case["wrap"],
                           diagonal=True)
        np.testing.assert_array_equal(got, np.array(case["labels"]), err_msg=str(case))
    # without the diagonals pixel 2 stays alone (the axis-only reading of the same frame)
    axis = oracle.label(rng, elev, az, 2.1, 1, wrap=True)
    assert axis[0, 2] == 2


def test_constant_is_the_angle_between_the_rays():
    g = np.random.default_rng(4)
    elev = np.sort(np.radians(g.uniform(-30, 30, 40)))[::-1]
    az = 2 * math.pi / 1024
    kd = oracle.tables_diag(elev, az, 6)
    for r in range(40):
        for k in range(1, 7):
            if r + k >= 40:
                assert kd[r, k - 1] == 0.0
                continue
            u1, u2 = _rays(elev, az, r, k)
            want = 2.0 - 2.0 * float(u1 @ u2)              # 2 - 2 cos(alpha)
            assert abs(kd[r, k - 1] - want) <= 1e-6 * want + 1e-12
            # Eq. 2 with this constant is the distance of the two points
            a, b = g.uniform(1, 60, 2)
            p1, p2 = a * u1, b * u2
            d2 = (a - b) ** 2 + float(kd[r, k - 1]) * a * b
            assert abs(d2 - float(np.sum((p1 - p2) ** 2))) <= 1e-5 * max(d2, 1e-3)


def _brute_labels(rng, elev, az, delta, S, wrap):
    """All pairs: adjacency straight from the definition, an independent fp32 predicate
    (numpy scalars), a depth-first search, minimum index per component."""
    R, C = rng.shape
    kv, kh = oracle.tables(elev, az, S)
    kd = oracle.tables_diag(elev, az, S)
    d2 = np.float32(delta) * np.float32(delta)
    valid = (rng > 0) & np.isfinite(rng)

    def pr(a, b, K):
        a, b, K = np.float32(a), np.float32(b), np.float32(K)
        with np.errstate(all="ignore"):
            t = np.float32(a - b)
            return bool(np.float32(np.float32(t * t) + np.float32(K * np.float32(a * b))) <= d2)

    def col_offsets(c1, c2):
        """Column offsets (signed, |o| = 1..S) that take column c1 to column c2."""
        out = []
        for k in range(1, S + 1):
            for sgn in (1, -1):
                c = c1 + sgn * k
                if wrap:
                    c %= C
                elif not 0 <= c < C:
                    continue
                if c == c2:
                    out.append(sgn * k)
        return out

    N = R * C
    adj = [[] for _ in range(N)]
    for p in range(N):
        for q in range(p + 1, N):
            r1, c1, r2, c2 = p // C, p % C, q // C, q % C
            if not (valid[r1, c1] and valid[r2, c2]):
                continue
            dr = r2 - r1
            ok = False
            if dr == 0:
                ok = any(pr(rng[r1, c1], rng[r2, c2], kh[r1, abs(o) - 1])
                         for o in col_offsets(c1, c2))
            elif 1 <= dr <= S:
                if c1 == c2:
                    ok = pr(rng[r1, c1], rng[r2, c2], kv[r1, dr - 1])
                if not ok and dr in [abs(o) for o in col_offsets(c1, c2)]:
                    ok = pr(rng[r1, c1], rng[r2, c2], kd[r1, dr - 1])
            if ok:
                adj[p].append(q)
                adj[q].append(p)
    lab = -np.ones(N, np.int64)
    for p in range(N):
        if lab[p] >= 0 or not valid[p // C, p % C]:
            continue
        stack = [p]
        lab[p] = p
        while stack:
            u = stack.pop()
            for v in adj[u]:
                if lab[v] < 0:
                    lab[v] = p
                    stack.append(v)
    return lab.reshape(R, C)


@pytest.mark.parametrize("seed", range(30))
def test_brute_force_tiny_grids(seed):
    g = np.random.default_rng(900 + seed)
    R, C, S = int(g.integers(1, 7)), int(g.integers(1, 7)), int(g.integers(1, 5))
    wrap = bool(g.integers(0, 2))
    vals = np.array([0.0, 1.0, 1.1, 1.3, 2.0, 6.0, np.nan, np.inf, -1.0], np.float32)
    rng = vals[g.integers(0, len(vals), (R, C))]
    elev = np.radians(np.linspace(25, -25, R)) if R > 1 else np.array([0.0])
    az = 2 * math.pi / max(C, 1) if g.integers(0, 2) else math.radians(4.0)
    delta = float(g.uniform(0.3, 2.5))
    got = oracle.label(rng, elev, az, delta, S, wrap=wrap, diagonal=True)
    np.testing.assert_array_equal(got, _brute_labels(rng, elev, az, delta, S, wrap))


def _edge_list(rng, elev, az, delta, S, wrap):
    """Every candidate pair of the frame, vectorised (numpy fp32), as (p, q) index arrays."""
    R, C = rng.shape
    kv, kh = oracle.tables(elev, az, S)
    kd = oracle.tables_diag(elev, az, S)
    d2 = np.float32(delta) * np.float32(delta)
    valid = (rng > 0) & np.isfinite(rng)
    rr, cc = np.meshgrid(np.arange(R), np.arange(C), indexing="ij")
    ps, qs = [], []

    def add(r2, c2, K):
        m = (r2 < R) & (c2 >= 0) & (c2 < C)
        r1s, c1s, r2s, c2s = rr[m], cc[m], r2[m], c2[m]
        Ks = K[m]
        a, b = rng[r1s, c1s], rng[r2s, c2s]
        with np.errstate(all="ignore"):
            t = (a - b).astype(np.float32)
            v = (t * t).astype(np.float32) + (Ks * (a * b).astype(np.float32)).astype(np.float32)
        ok = valid[r1s, c1s] & valid[r2s, c2s] & (v.astype(np.float32) <= d2)
        ps.append(r1s[ok] * C + c1s[ok])
        qs.append(r2s[ok] * C + c2s[ok])

    for k in range(1, S + 1):
        ch = cc + k
        ch = ch % C if wrap else ch
        add(rr, ch, np.broadcast_to(kh[:, k - 1:k], (R, C)))
        add(rr + k, cc, np.broadcast_to(kv[:, k - 1:k], (R, C)))
        for sgn in (1, -1):
            cd = cc + sgn * k
            cd = cd % C if wrap else cd
            add(rr + k, cd, np.broadcast_to(kd[:, k - 1:k], (R, C)))
    return np.concatenate(ps), np.concatenate(qs)


@pytest.mark.parametrize("S,wrap", [(1, True), (2, False), (3, True), (5, True), (5, False)])
def test_connected_components_of_an_independent_edge_list(S, wrap):
    scipy_sparse = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = np.random.default_rng(31 + S)
    R, C = 40, 96
    base = 6 + 2 * np.sin(np.arange(C) / 9.0)[None, :] + 0.04 * np.arange(R)[:, None]
    rng = (base + g.normal(0, 0.08, (R, C))).astype(np.float32)
    rng[g.random((R, C)) < 0.3] = 0
    elev = np.radians(np.linspace(12, -12, R))
    az = 2 * math.pi / C
    p, q = _edge_list(rng, elev, az, 0.35, S, wrap)
    N = R * C
    A = scipy_sparse.coo_matrix((np.ones(len(p)), (p, q)), shape=(N, N))
    _, comp = csgraph.connected_components(A, directed=False)
    valid = ((rng > 0) & np.isfinite(rng)).reshape(-1)
    mins = np.full(comp.max() + 1, N)
    np.minimum.at(mins, comp, np.arange(N))
    want = np.where(valid, mins[comp], -1).reshape(R, C)
    got = oracle.label(rng, elev, az, 0.35, S, wrap=wrap, diagonal=True)
    np.testing.assert_array_equal(got, want)


def test_partitions_nest():
    """Every component without the diagonals lies inside one component with them, and the
    diagonals do join something on a noisy frame."""
    g = np.random.default_rng(8)
    R, C = 32, 128
    rng = (8 + g.normal(0, 0.2, (R, C))).astype(np.float32)
    rng[g.random((R, C)) < 0.35] = 0
    elev = np.radians(np.linspace(10, -10, R))
    az = 2 * math.pi / C
    for S in (1, 3):
        a = oracle.label(rng, elev, az, 0.4, S)
        d = oracle.label(rng, elev, az, 0.4, S, diagonal=True)
        m = a >= 0
        assert np.array_equal(m, d >= 0)
        rep = {}
        for la, ld in zip(a[m], d[m]):
            assert rep.setdefault(int(la), int(ld)) == ld
        assert len(np.unique(d[m])) < len(np.unique(a[m]))


def test_not_combined_with_the_sparse_map():
    with pytest.raises(ValueError):
        oracle.label(np.ones((2, 4), np.float32), np.array([0.1, 0.0]), 1.0, 0.5, 2,
                     lattice=True, diagonal=True)
