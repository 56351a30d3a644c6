"""GPU parity of flic_edges in both of its forms — the 16-byte word pass (cols % 4 == 0,
aligned buffers, no ground filter) and the one-pixel-per-thread pass (every other frame) —
bit for bit against oracle.edges: every skip 1..8, wrap and no wrap, the sparse Map
Connection, rows fewer than, equal to and just past a thread's row tile, rows of one word,
widths that wrap several times within the offsets, invalid readings of every kind, and
buffers offset from their 16-byte boundary."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


def _frame(seed, R, C):
    g = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        base = 5 + 3 * np.sin(np.arange(C) / 7.0)[None, :] + 0.05 * np.arange(R)[:, None]
        rng = base + g.normal(0, 0.05, (R, C))
        rng[g.random((R, C)) < 0.15] = 0
    elif kind == 1:
        vals = np.array([0.0, 1.0, 1.2, 2.0, 2.1, 7.0, np.nan, np.inf, -np.inf, -3.0, 3.4e38])
        rng = vals[g.integers(0, len(vals), (R, C))]
    else:
        rng = g.uniform(0.5, 30, (R, C))
        rng[g.random((R, C)) < 0.3] = 0
    elev = np.radians(np.linspace(12, -12, R)) if R > 1 else np.array([0.0])
    return rng.astype(np.float32), elev, 2 * math.pi / C, float(np.float32(g.uniform(0.2, 1.5)))


def _edges(flic, rng, elev, az, delta, S, wrap, lattice, offset=0):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, S, wrap=wrap, lattice=lattice)
    try:
        # offset > 0: the frame starts `offset` floats (and the mask `offset` uint16) past
        # an allocation's 16-byte boundary
        rbuf = torch.zeros(R * C + offset, dtype=torch.float32, device=DEV)
        rbuf[offset:] = torch.from_numpy(rng.reshape(-1)).to(DEV)
        mbuf = torch.full((R * C + offset,), -1, dtype=torch.int16, device=DEV)
        flic.flic_edges(h, rbuf.data_ptr() + 4 * offset, mbuf.data_ptr() + 2 * offset)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        m = mbuf.cpu().numpy().view(np.uint16)
        assert np.all(m[:offset] == 0xFFFF)
        return m[offset:].reshape(R, C)
    finally:
        h.close()


SHAPES = [(1, 4), (1, 8), (2, 12), (3, 4), (4, 16), (5, 20), (7, 1024), (8, 1800), (9, 36),
          (16, 1800), (33, 2048), (64, 2048), (130, 44), (3, 6), (5, 1022), (6, 1801)]


@pytest.mark.parametrize("S", range(1, 9))
@pytest.mark.parametrize("wrap", [True, False])
def test_every_skip_and_shape(flic, S, wrap):
    for i, (R, C) in enumerate(SHAPES):
        rng, elev, az, delta = _frame(1000 * S + 10 * i + wrap, R, C)
        got = _edges(flic, rng, elev, az, delta, S, wrap, False)
        want = oracle.edges(rng, elev, az, delta, S, wrap)
        np.testing.assert_array_equal(got, want, err_msg=f"{R}x{C} S{S} wrap={wrap}")


@pytest.mark.parametrize("S", [2, 3, 5, 8])
def test_sparse_map_connection(flic, S):
    for i, (R, C) in enumerate([(4, 16), (9, 36), (33, 2048), (17, 1800), (6, 1801)]):
        for wrap in (True, False):
            rng, elev, az, delta = _frame(7000 + 10 * S + i, R, C)
            got = _edges(flic, rng, elev, az, delta, S, wrap, True)
            want = oracle.edges(rng, elev, az, delta, S, wrap, lattice=True)
            np.testing.assert_array_equal(got, want, err_msg=f"{R}x{C} S{S} wrap={wrap}")


@pytest.mark.parametrize("offset", [1, 2, 3, 4])
def test_buffers_off_their_boundary(flic, offset):
    """offset 1-3 floats leaves the range image off 16 bytes (and offsets 1-3 leave the mask
    off 8 bytes): the one-pixel pass; offset 4 is aligned again: the word pass."""
    rng, elev, az, delta = _frame(40 + offset, 24, 2048)
    got = _edges(flic, rng, elev, az, delta, 5, True, False, offset=offset)
    np.testing.assert_array_equal(got, oracle.edges(rng, elev, az, delta, 5, True))


def test_largest_frame(flic):
    R, C = 512, 4096
    rng, elev, az, delta = _frame(77, R, C)
    for S in (1, 3, 8):
        got = _edges(flic, rng, elev, az, delta, S, True, False)
        np.testing.assert_array_equal(got, oracle.edges(rng, elev, az, delta, S, True))
