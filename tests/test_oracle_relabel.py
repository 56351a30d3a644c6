"""Pins of the oracle's cluster-candidate filter and compact numbering (§III-B)."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _hand():
    with open(os.path.join(HERE, "golden", "relabel_hand_3x4.json")) as fh:
        return json.load(fh)


def test_hand_fixture():
    g = _hand()
    for case in g["cases"]:
        out, n = oracle.filter_relabel(np.array(g["labels"]), case["min_size"])
        assert n == case["count"]
        assert out.tolist() == case["out"]


def test_hand_fixture_from_the_labeller():
    """The fixture's input is what the oracle's own labeller gives on the hand frame."""
    with open(os.path.join(HERE, "golden", "hand_3x4.json")) as fh:
        h = json.load(fh)
    lab = oracle.label(np.array(h["range"], np.float32), np.radians(h["elevation_deg"]),
                       np.radians(h["az_step_deg"]), 2.1, 1, True)
    assert lab.reshape(3, 4).tolist() == _hand()["labels"]


def _grid(rows, cols, p, seed):
    g = np.random.default_rng(seed)
    valid = g.random((rows, cols)) < p
    rng = np.where(valid, 5.0, 0.0).astype(np.float32)
    return rng, valid


@pytest.mark.parametrize("seed", range(6))
def test_numbering_is_scipys(seed):
    """S=1 without wrap and a threshold every pair passes: components are the 4-connected
    components of the measurements, and scipy.ndimage.label numbers them 1..N in the
    raster order of their first pixel, i.e. ours + 1 (§III-B-1 uses that function)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng, valid = _grid(17, 23, 0.55, seed)
    elev = np.radians(np.linspace(10, -10, 17))
    lab = oracle.label(rng, elev, 2 * np.pi / 23, 100.0, 1, False).reshape(17, 23)
    ours, n = oracle.filter_relabel(lab, 1)
    ref, nref = ndimage.label(valid)
    assert n == nref
    assert np.array_equal(ours + 1, ref)


@pytest.mark.parametrize("seed", range(6))
def test_sizes_by_brute_force(seed):
    """Kept components are exactly those with at least min_size pixels, counted one pixel
    at a time; ids are contiguous and follow the order of the components' first pixels."""
    rng, valid = _grid(13, 19, 0.6, 100 + seed)
    elev = np.radians(np.linspace(10, -10, 13))
    lab = oracle.label(rng, elev, 2 * np.pi / 19, 100.0, 1, False).reshape(13, 19)
    for m in (0, 1, 2, 3, 5, 8):
        ours, n = oracle.filter_relabel(lab, m)
        size = {}
        first = {}
        for i, l in enumerate(lab.reshape(-1).tolist()):
            if l >= 0:
                size[l] = size.get(l, 0) + 1
                first.setdefault(l, i)
        kept = sorted((first[l], l) for l in size if size[l] >= m)
        assert n == len(kept)
        want = {l: k for k, (_, l) in enumerate(kept)}
        for i, (l, o) in enumerate(zip(lab.reshape(-1).tolist(), ours.reshape(-1).tolist())):
            assert o == (want[l] if l >= 0 and l in want else -1), (m, i)


def test_degenerate():
    empty = np.full((4, 5), -1)
    out, n = oracle.filter_relabel(empty, 1)
    assert n == 0 and (out == -1).all()
    one = np.zeros((2, 3), np.int64)  # one component of six pixels, minimum 0
    assert oracle.filter_relabel(one, 6)[1] == 1
    assert oracle.filter_relabel(one, 7)[1] == 0
    assert oracle.filter_relabel(one, -3)[1] == 1
