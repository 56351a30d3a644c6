"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself:
  - the paper's printed maximum-range figures (§III-B) -> angle units and K-table formula
  - the hand-worked 3x4 frame (tests/golden/hand_3x4.json) -> edges, wrap, skip, ties
  - brute force on tiny grids: all ordered pairs, an independent fp32 predicate, DFS
  - scipy.ndimage.label on the paper's interleaved "supersize" image (§III-B-1) for S = 1
  - scipy.sparse.csgraph.connected_components on an independently built edge list
  - invariants: symmetry, min-index labels, coarsening in S and delta
  - the FP64 decision (Eq. 2 in double): flips only within 1e-5 m of delta
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from paper_2003_00575_gb300 import synth

F32 = np.float32


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- paper-printed numbers

def _largest_connected_range(vertical: bool, alpha_deg: float, delta: float) -> float:
    """Bisect the largest equal range R whose two readings the oracle connects."""
    a = math.radians(alpha_deg)
    if vertical:
        elev = np.array([0.0, a])
        az = math.radians(0.2)
    else:
        elev = np.array([0.0, math.radians(2.0)])
        az = a

    def connected(R):
        img = np.zeros((2, 3), np.float32)
        if vertical:
            img[0, 0] = img[1, 0] = R
            bit = 1 << 8
        else:
            img[0, 0] = img[0, 1] = R
            bit = 1
        m = oracle.edges(img, elev, az, delta, 1, wrap=False)
        return bool(m[0, 0] & bit)

    lo, hi = 1.0, 2000.0
    assert connected(lo) and not connected(hi)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if connected(mid):
            lo = mid
        else:
            hi = mid
    return lo


def test_max_range_matches_paper(golden_dir):
    g = _golden(golden_dir, "max_range.json")
    for key, vertical in (("vertical", True), ("horizontal", False)):
        spec = g[key]
        r_star = _largest_connected_range(vertical, spec["alpha_deg"], g["delta"])
        assert round(r_star, spec["decimals"]) == pytest.approx(spec["printed_max_range_m"]), \
            (key, r_star)


def test_max_range_edge_just_inside_and_outside():
    elev = np.array([0.0, math.radians(0.4)])
    for R, want in ((114.58, True), (114.60, False)):
        img = np.zeros((2, 2), np.float32)
        img[:, 0] = R
        m = oracle.edges(img, elev, math.radians(0.09), 0.8, 1, wrap=False)
        assert bool(m[0, 0] & (1 << 8)) == want, R


# ---------------------------------------------------------------- hand-worked example

def test_hand_example(golden_dir):
    g = _golden(golden_dir, "hand_3x4.json")
    elev = np.radians(g["elevation_deg"])
    az = math.radians(g["az_step_deg"])
    rng = np.array(g["range"], np.float32)
    kv, kh = oracle.tables(elev, az, g["tables"]["skip"])
    np.testing.assert_array_equal(kv, np.array(g["tables"]["Kv"], np.float32))
    np.testing.assert_array_equal(kh, np.array(g["tables"]["Kh"], np.float32))
    for case in g["cases"]:
        lab = oracle.label(rng, elev, az, case["delta"], case["skip"], wrap=case["wrap"])
        np.testing.assert_array_equal(lab, np.array(case["labels"]), err_msg=str(case))
        if "edges" in case:
            m = oracle.edges(rng, elev, az, case["delta"], case["skip"], wrap=case["wrap"])
            np.testing.assert_array_equal(m, np.array(case["edges"]), err_msg=str(case))


# ---------------------------------------------------------------- independent fp32 predicate

def _pred32(a, b, K, delta):
    """Eq. 2/3 in numpy float32 scalars: each operation rounded to fp32 on its own."""
    a, b, K, d = F32(a), F32(b), F32(K), F32(delta)
    t = F32(a - b)
    d2 = F32(F32(t * t) + F32(K * F32(a * b)))
    return bool(d2 <= F32(d * d))


def _valid(x):
    return bool(np.isfinite(x) and x > 0)


def _brute_pairs(rng, kv, kh, S, delta, wrap):
    """All unordered pairs {p, q} joined by an edge, by enumerating every ordered pair and
    every offset and asking whether q is p's k-th right or lower neighbour."""
    R, C = rng.shape
    N = R * C
    E = set()
    for p, q in itertools.permutations(range(N), 2):
        rp, cp = divmod(p, C)
        rq, cq = divmod(q, C)
        a, b = rng[rp, cp], rng[rq, cq]
        if not (_valid(a) and _valid(b)):
            continue
        for k in range(1, S + 1):
            right = (rq == rp) and ((cq == (cp + k) % C) if wrap else (cq == cp + k))
            down = (cq == cp) and (rq == rp + k)
            if right and _pred32(a, b, kh[rp, k - 1], delta):
                E.add((min(p, q), max(p, q)))
            if down and _pred32(a, b, kv[rp, k - 1], delta):
                E.add((min(p, q), max(p, q)))
    return E


def _dfs_labels(rng, E):
    R, C = rng.shape
    N = R * C
    adj = {p: [] for p in range(N)}
    for p, q in E:
        adj[p].append(q)
        adj[q].append(p)
    lab = -np.ones(N, np.int64)
    for p in range(N):
        if lab[p] != -1 or not _valid(rng.flat[p]):
            continue
        comp, stack = [], [p]
        lab[p] = p
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in adj[u]:
                if lab[v] == -1:
                    lab[v] = p
                    stack.append(v)
        m = min(comp)
        for u in comp:
            lab[u] = m
    return lab.reshape(R, C)


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_tiny(seed):
    g = np.random.default_rng(1000 + seed)
    R = int(g.integers(1, 7))
    C = int(g.integers(1, 7))
    S = int(g.integers(1, 5))
    wrap = bool(g.integers(0, 2))
    # few distinct values so that ties, invalid cells and long skips all occur
    vals = np.array([0.0, 1.0, 1.5, 2.0, 3.0, 5.0, np.nan, np.inf, -1.0], np.float32)
    rng = vals[g.integers(0, len(vals), (R, C))]
    elev = np.sort(g.uniform(-0.6, 0.6, R))[::-1] if R > 1 else np.array([0.0])
    az = float(g.uniform(0.2, 1.6))
    delta = float(F32(g.uniform(0.5, 3.0)))
    kv, kh = oracle.tables(elev, az, S)
    E = _brute_pairs(rng, kv, kh, S, delta, wrap)
    want = _dfs_labels(rng, E)
    got = oracle.label(rng, elev, az, delta, S, wrap=wrap)
    np.testing.assert_array_equal(got, want)
    # edge bits agree with the pair set (bit k-1 right, 8+k-1 down)
    m = oracle.edges(rng, elev, az, delta, S, wrap=wrap)
    E2 = set()
    for p in range(R * C):
        r, c = divmod(p, C)
        for k in range(1, S + 1):
            if m[r, c] & (1 << (k - 1)):
                q = r * C + (((c + k) % C) if wrap else c + k)
                if q != p:
                    E2.add((min(p, q), max(p, q)))
            if m[r, c] & (1 << (8 + k - 1)):
                q = (r + k) * C + c
                E2.add((min(p, q), max(p, q)))
    assert E2 == {e for e in E if e[0] != e[1]}


# ---------------------------------------------------------------- library special cases

def _edge_arrays(rng, kv, kh, S, delta, wrap):
    """Vectorised independent edge list (numpy float32 elementwise, each op rounded)."""
    R, C = rng.shape
    d2max = F32(delta) * F32(delta)
    valid = np.isfinite(rng) & (rng > 0)
    P, Q = [], []
    idx = np.arange(R * C).reshape(R, C)
    for k in range(1, S + 1):
        # horizontal
        if wrap:
            b = np.roll(rng, -k, axis=1)
            vb = np.roll(valid, -k, axis=1)
            qi = np.roll(idx, -k, axis=1)
            a, va, pi, K = rng, valid, idx, kh[:, k - 1][:, None]
        else:
            if k >= C:
                continue
            a, b = rng[:, :-k], rng[:, k:]
            va, vb = valid[:, :-k], valid[:, k:]
            pi, qi = idx[:, :-k], idx[:, k:]
            K = kh[:, k - 1][:, None]
        t = (a - b).astype(F32)
        d2 = (t * t).astype(F32) + (K.astype(F32) * (a * b).astype(F32)).astype(F32)
        ok = va & vb & (d2.astype(F32) <= d2max)
        P.append(pi[ok]); Q.append(qi[ok])
        # vertical
        if k < R:
            a, b = rng[:-k], rng[k:]
            K = kv[:-k, k - 1][:, None].astype(F32)
            t = (a - b).astype(F32)
            d2 = (t * t).astype(F32) + (K * (a * b).astype(F32)).astype(F32)
            ok = valid[:-k] & valid[k:] & (d2.astype(F32) <= d2max)
            P.append(idx[:-k][ok]); Q.append(idx[k:][ok])
    return np.concatenate(P) if P else np.zeros(0, int), np.concatenate(Q) if Q else np.zeros(0, int)


def _min_index_labels(comp_ids, valid_flat):
    N = comp_ids.shape[0]
    lab = -np.ones(N, np.int64)
    first = {}
    for p in range(N):
        if not valid_flat[p]:
            continue
        c = comp_ids[p]
        if c not in first:
            first[c] = p
        lab[p] = first[c]
    return lab


def _crop(frame, rows, cols, r0=0, c0=0):
    rng = frame.range[r0:r0 + rows, c0:c0 + cols].copy()
    elev = frame.sensor.elevation[r0:r0 + rows]
    return rng, elev


def test_supersize_ndimage_label_s1_no_wrap():
    """§III-B-1: with S = 1 and no wrap, 4-connected labelling of the interleaved image
    (measurement, horizontal-connection, vertical-connection cells) gives the clusters."""
    f = synth.config_c1()
    for c0 in (0, 300, 900):
        rng, elev = _crop(f, 16, 120, 0, c0)
        R, C = rng.shape
        kv, kh = oracle.tables(elev, f.sensor.az_step, 1)
        P, Q = _edge_arrays(rng, kv, kh, 1, f.delta, wrap=False)
        sup = np.zeros((2 * R, 2 * C), np.uint8)
        valid = np.isfinite(rng) & (rng > 0)
        sup[0::2, 0::2] = valid
        for p, q in zip(P, Q):
            rp, cp = divmod(int(p), C)
            rq, cq = divmod(int(q), C)
            sup[rp + rq, cp + cq] = 1  # midpoint cell of the interleaved image
        lab_sup, _ = ndi.label(sup)  # default structure: 4-connectivity
        comp = lab_sup[0::2, 0::2].reshape(-1)
        want = _min_index_labels(comp, valid.reshape(-1)).reshape(R, C)
        got = oracle.label(rng, elev, f.sensor.az_step, f.delta, 1, wrap=False)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("which,skip,wrap", [("c2", 3, True), ("c3", 5, True), ("c2", 2, False),
                                             ("c3", 1, True)])
def test_csgraph_components(which, skip, wrap):
    f = synth.config_c2() if which == "c2" else synth.config_c3(with_xyz=False)
    rng, elev = _crop(f, 24, f.sensor.cols, 8, 0)  # full width so the wrap seam is real
    R, C = rng.shape
    kv, kh = oracle.tables(elev, f.sensor.az_step, skip)
    P, Q = _edge_arrays(rng, kv, kh, skip, f.delta, wrap)
    A = coo_matrix((np.ones(P.shape[0]), (P, Q)), shape=(R * C, R * C))
    _, comp = connected_components(A, directed=False)
    valid = (np.isfinite(rng) & (rng > 0)).reshape(-1)
    want = _min_index_labels(comp, valid).reshape(R, C)
    got = oracle.label(rng, elev, f.sensor.az_step, f.delta, skip, wrap=wrap)
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- invariants

def test_pred_symmetric_and_matches_independent():
    g = np.random.default_rng(7)
    a = g.uniform(0.1, 120, 4000).astype(F32)
    b = (a + g.normal(0, 0.5, 4000)).astype(F32)
    K = g.uniform(1e-7, 1e-2, 4000).astype(F32)
    for x, y, k in zip(a[:800], b[:800], K[:800]):
        assert oracle.pred(x, y, k, 0.5) == oracle.pred(y, x, k, 0.5)
        assert oracle.pred(x, y, k, 0.5) == _pred32(x, y, k, 0.5)


def _partition_refines(fine, coarse):
    """Every pair joined in `fine` is joined in `coarse`."""
    m = fine >= 0
    assert np.array_equal(m, coarse >= 0)
    f, c = fine[m], coarse[m]
    # each fine component maps to exactly one coarse component
    order = np.argsort(f, kind="stable")
    fs, cs = f[order], c[order]
    starts = np.r_[0, np.flatnonzero(np.diff(fs)) + 1]
    for s, e in zip(starts, np.r_[starts[1:], fs.shape[0]]):
        assert np.all(cs[s:e] == cs[s])


def test_invariants_on_synthetic_frames():
    f = synth.config_c2()
    rng, elev, az = f.range, f.sensor.elevation, f.sensor.az_step
    prev = None
    for S in range(1, 6):
        lab = oracle.label(rng, elev, az, 0.5, S)
        flat = lab.reshape(-1)
        idx = np.arange(flat.shape[0])
        valid = (np.isfinite(rng) & (rng > 0)).reshape(-1)
        assert np.array_equal(flat >= 0, valid)
        assert np.all(flat[valid] <= idx[valid])           # label is a member's index ...
        assert np.all(flat[flat[valid]] == flat[valid])    # ... the minimum one (a fixed point)
        # every edge joins equal labels
        m = oracle.edges(rng, elev, az, 0.5, S)
        R, C = rng.shape
        for k in range(1, S + 1):
            rr, cc = np.nonzero(m & (1 << (k - 1)))
            assert np.all(lab[rr, cc] == lab[rr, (cc + k) % C])
            rr, cc = np.nonzero(m & (1 << (8 + k - 1)))
            assert np.all(lab[rr, cc] == lab[rr + k, cc])
        if prev is not None:
            _partition_refines(prev, lab)
        prev = lab
    fine = oracle.label(rng, elev, az, 0.3, 2)
    coarse = oracle.label(rng, elev, az, 0.6, 2)
    _partition_refines(fine, coarse)


# ---------------------------------------------------------------- fp32 vs fp64

@pytest.mark.parametrize("which", ["c1", "c2", "c3"])
def test_fp64_flips_only_near_threshold(which):
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[which]()
    pairs, flips, worst = oracle.flips(f.range, f.sensor.elevation, f.sensor.az_step, f.delta,
                                       f.skip)
    assert pairs > 10_000
    assert flips == 0 or worst < 1e-5


def test_fp64_flips_near_ties():
    """Pairs built to sit within ~1e-6 m (half) or ~5e-4 m (half) of delta at 5-110 m: any
    fp32/fp64 disagreement
    must lie within 1e-5 m of delta, while the literal Eq. 3 form (two d^2 terms cancelling)
    disagrees further out."""
    g = np.random.default_rng(11)
    n = 3000
    delta = F32(0.5)
    alpha = math.radians(0.2)
    rows = []
    for i in range(n):
        a = g.uniform(5, 110)
        # solve D(a, b) = delta for b > a (law of cosines), then nudge by ~1e-6 m
        c = math.cos(alpha)
        b = a * c + math.sqrt(max(float(delta) ** 2 - (a * math.sin(alpha)) ** 2, 0.0))
        b += g.uniform(-2e-6, 2e-6) if i % 2 == 0 else g.uniform(-5e-4, 5e-4)
        rows.append((a, b))
    img = np.array(rows, np.float32).T.copy()  # 2 rows x n cols: vertical pairs
    elev = np.array([0.0, alpha])
    pairs, flips, worst = oracle.flips(img, elev, 2 * math.pi / n, float(delta), 1, wrap=False)
    assert flips == 0 or worst < 1e-5
    # the literal form: count decisions that disagree with fp64 by more than 1e-5 m
    C2 = F32(2.0 * math.cos(alpha))
    far = 0
    for a, b in zip(img[0], img[1]):
        D = math.sqrt((float(a) - float(b)) ** 2 + 4 * float(a) * float(b) * math.sin(alpha / 2) ** 2)
        if oracle.pred_paper_form(a, b, C2, float(delta)) != (D <= float(delta)) \
                and abs(D - float(delta)) >= 1e-5:
            far += 1
    assert far > 0


def test_frame_flips_of_the_literal_form():
    """oracle.flips_paper_form counts the same candidate pairs as oracle.flips and decides
    each by the scalar literal-form predicate (checked pair by pair on a small frame); on
    c3 the literal form of Eq. 3 flips decisions further than 1e-5 m from delta, the
    cancellation-free form none."""
    g = np.random.default_rng(12)
    R, C, S = 6, 40, 3
    rng = (g.uniform(20.0, 90.0, (R, C))).astype(np.float32)
    rng[g.random((R, C)) < 0.2] = 0.0
    elev = np.radians(np.linspace(10.0, -10.0, R))
    az = 2 * math.pi / C
    delta = 2.5
    pairs, flips, far, dev = oracle.flips_paper_form(rng, elev, az, delta, S)
    want_pairs = want_flips = 0
    for r in range(R):
        for c in range(C):
            a = rng[r, c]
            if not a > 0:
                continue
            for k in range(1, S + 1):
                for rr, cc, alpha in ((r + k, c, abs(elev[min(r + k, R - 1)] - elev[r])),
                                      (r, (c + k) % C, k * az)):
                    if rr >= R or not rng[rr, cc] > 0:
                        continue
                    b = rng[rr, cc]
                    want_pairs += 1
                    f32 = oracle.pred_paper_form(a, b, float(np.float32(2 * math.cos(alpha))),
                                                 delta)
                    D = math.sqrt((float(a) - float(b)) ** 2
                                  + 4 * float(a) * float(b) * math.sin(alpha / 2) ** 2)
                    want_flips += f32 != (D <= delta)
    assert (pairs, flips) == (want_pairs, want_flips)
    from paper_2003_00575_gb300 import synth
    f = synth.config_c3(with_xyz=False)
    p, n, d = oracle.flips(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
    p2, n2, far2, d2 = oracle.flips_paper_form(f.range, f.sensor.elevation, f.sensor.az_step,
                                               f.delta, f.skip)
    assert p == p2 and n == 0 and far2 > 0 and d2 >= 1e-5
