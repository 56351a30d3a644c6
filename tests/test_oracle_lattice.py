"""Pins of the oracle's sparse Map Connection (§III-B-2): direct neighbours of every pixel,
plus offset S only from the sub-lattice of every S-th row and column (oracle.label /
oracle.edges with lattice=True).  Checked against the paper's own construction (the three
binary images arranged as in Fig. 2 and labelled with 4-connectivity, here by scipy), a
hand-worked case, brute force, and the nesting of the edge sets."""
import json
import os

import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_hand_4x6.json")


def _same_partition(a, b):
    """Two label images describe the same components (and the same invalid pixels)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    assert np.array_equal(a < 0, b < 0)
    m = a >= 0
    pairs = set(zip(a[m].tolist(), b[m].tolist()))
    return len(pairs) == len(set(a[m].tolist())) == len(set(b[m].tolist()))


def test_hand_case():
    g = json.load(open(GOLDEN))
    rng = np.array(g["range"], np.float32).reshape(g["rows"], g["cols"])
    args = (rng, np.array(g["elevation"]), g["az_step"], g["delta"], g["skip"], g["wrap"])
    assert oracle.label(*args, lattice=True).reshape(-1).tolist() == g["labels_lattice"]
    assert oracle.label(*args).reshape(-1).tolist() == g["labels_offsets_1_to_2"]
    assert oracle.label(rng, *args[1:4], 1, g["wrap"]).reshape(-1).tolist() == g["labels_s1"]


def _frame(seed, R, C, n, p=0.8):
    g = np.random.default_rng(seed)
    rng = g.uniform(4.0, 6.0, (R, C)).astype(np.float32)
    rng[g.random((R, C)) > p] = 0.0
    elev = np.radians(np.linspace(12.0, -12.0, R)) if R > 1 else np.array([0.0])
    return rng, elev, 2 * np.pi / C, float(g.uniform(0.2, 0.7))


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("n", [2, 3, 4])
def test_paper_construction_on_the_sub_lattice(seed, n):
    """Readings only at lattice points: no direct pair exists, so the components are those
    of the every-n-th-point map, which the paper builds as a small range image whose
    horizontal and vertical threshold images are arranged with it (Fig. 2) and labelled
    with 4-connectivity."""
    R, C = 3 * n + 2, 5 * n + 1
    rng, elev, az, delta = _frame(seed, R, C, n)
    keep = np.zeros((R, C), bool)
    keep[::n, ::n] = True
    rng[~keep] = 0.0
    got = oracle.label(rng, elev, az, delta, n, wrap=False, lattice=True)
    # the paper's construction on the sub-sampled image, with the angle of offset n
    kv, kh = oracle.tables(elev, az, n)
    sub = rng[::n, ::n]
    rs, cs = sub.shape
    big = np.zeros((2 * rs - 1, 2 * cs - 1), bool)
    for i in range(rs):
        for j in range(cs):
            a = float(sub[i, j])
            big[2 * i, 2 * j] = a > 0
            if j + 1 < cs and a > 0 and sub[i, j + 1] > 0:
                big[2 * i, 2 * j + 1] = oracle.pred(a, float(sub[i, j + 1]), kh[i * n, n - 1], delta)
            if i + 1 < rs and a > 0 and sub[i + 1, j] > 0:
                big[2 * i + 1, 2 * j] = oracle.pred(a, float(sub[i + 1, j]), kv[i * n, n - 1], delta)
    lab, _ = scipy_ndimage.label(big)  # 4-connectivity
    want = np.full((R, C), -1, np.int64)
    want[::n, ::n] = np.where(lab[::2, ::2] > 0, lab[::2, ::2], -1)
    assert _same_partition(got, want)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("wrap", [False, True])
def test_spacing_one_and_nesting(seed, wrap):
    """S = 1 lattice is the plain 4-neighbourhood; the lattice's pairs lie between the
    direct pairs and the pairs of offsets 1..S, so its components refine the latter's and
    are refined by the former's."""
    R, C = 13, 29
    rng, elev, az, delta = _frame(100 + seed, R, C, 3, p=0.65)
    s1 = oracle.label(rng, elev, az, delta, 1, wrap)
    assert np.array_equal(oracle.label(rng, elev, az, delta, 1, wrap, lattice=True), s1)
    for n in (2, 3, 5):
        lat = oracle.label(rng, elev, az, delta, n, wrap, lattice=True).reshape(-1)
        full = oracle.label(rng, elev, az, delta, n, wrap).reshape(-1)
        s1f = s1.reshape(-1)
        m = s1f >= 0
        # each S = 1 component inside one lattice component, each lattice one inside one
        # component of offsets 1..n
        assert len(set(zip(s1f[m].tolist(), lat[m].tolist()))) == len(set(s1f[m].tolist()))
        assert len(set(zip(lat[m].tolist(), full[m].tolist()))) == len(set(lat[m].tolist()))


def _brute(rng, elev, az, delta, n, wrap):
    """Union-find over the explicit pair list of the sparse map."""
    R, C = rng.shape
    kv, kh = oracle.tables(elev, az, n)
    par = list(range(R * C))

    def find(x):
        while par[x] != x:
            x = par[x]
        return x

    for r in range(R):
        for c in range(C):
            if not rng[r, c] > 0:
                continue
            for k in range(1, n + 1):
                if k != 1 and not (k == n and r % n == 0 and c % n == 0):
                    continue
                targets = []
                cc = c + k
                if cc < C or wrap:
                    targets.append((r, cc % C, kh[r, k - 1]))
                if r + k < R:
                    targets.append((r + k, c, kv[r, k - 1]))
                for rr, c2, K in targets:
                    b = rng[rr, c2]
                    if b > 0 and oracle.pred(float(rng[r, c]), float(b), float(K), delta):
                        x, y = find(r * C + c), find(rr * C + c2)
                        if x != y:
                            par[max(x, y)] = min(x, y)
    out = np.full(R * C, -1, np.int64)
    for p in range(R * C):
        if rng.reshape(-1)[p] > 0:
            out[p] = find(p)
    return out


@pytest.mark.parametrize("seed", range(8))
def test_brute_force(seed):
    g = np.random.default_rng(500 + seed)
    R, C, n = int(g.integers(1, 9)), int(g.integers(2, 14)), int(g.integers(2, 5))
    rng, elev, az, delta = _frame(600 + seed, R, C, n, p=0.7)
    wrap = bool(seed % 2)
    got = oracle.label(rng, elev, az, delta, n, wrap, lattice=True).reshape(-1)
    assert np.array_equal(got, _brute(rng, elev, az, delta, n, wrap))  # both: min index


def test_edges_follow_the_rule():
    rng, elev, az, delta = _frame(7, 9, 17, 3, p=1.0)
    full = oracle.edges(rng, elev, az, 3.0, 3, True)   # large delta: every pair an edge
    lat = oracle.edges(rng, elev, az, 3.0, 3, True, lattice=True)
    R, C = rng.shape
    for r in range(R):
        for c in range(C):
            allowed = 0x1 | 0x100
            if r % 3 == 0 and c % 3 == 0:
                allowed |= (1 << 2) | (1 << (8 + 2))
            assert lat[r, c] == full[r, c] & allowed, (r, c)
