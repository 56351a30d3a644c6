"""GPU parity of the sparse Map Connection (FLIC_FLAG_SUBLATTICE, §III-B-2: direct
neighbours of every pixel, offset S only from every S-th row and column): flic_label,
flic_label_batch and flic_edges element by element against oracle.label / oracle.edges
with lattice=True, over many strip layouts (the border merge applies the same rule)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2003_00575_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


def _check(flic, rng, elev, az, delta, S, wrap, tuning=None, ground=None):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, S, wrap=wrap, lattice=True)
    try:
        if tuning:
            flic.flic_set_tuning(h, *tuning)
        src = np.ascontiguousarray(rng, np.float32)
        if ground:
            flic.flic_set_ground(h, *ground)
            g = oracle.ground(src, elev, *ground)
            src_o = np.where(g, np.float32(0), src)
        else:
            src_o = src
        r = torch.from_numpy(src).to(DEV)
        lab = torch.full((R * C,), 777, dtype=torch.int32, device=DEV)
        m = torch.zeros(R * C, dtype=torch.int16, device=DEV)
        flic.flic_label(h, r, lab)
        flic.flic_edges(h, r, m)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        want = oracle.label(src_o, elev, az, delta, S, wrap, lattice=True)
        np.testing.assert_array_equal(lab.cpu().numpy().reshape(R, C), want)
        np.testing.assert_array_equal(m.cpu().numpy().view(np.uint16).reshape(R, C),
                                      oracle.edges(src_o, elev, az, delta, S, wrap, lattice=True))
        return want
    finally:
        h.close()


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
@pytest.mark.parametrize("S", [2, 3, 5])
def test_configs(flic, name, S):
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[name]()
    want = _check(flic, f.range, f.sensor.elevation, f.sensor.az_step, f.delta, S, True)
    full = oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, S)
    s1 = oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, 1)
    # the sparse map lies between the direct neighbourhood and offsets 1..S
    n = lambda x: len(np.unique(x[x >= 0]))  # noqa: E731
    assert n(full) <= n(want) <= n(s1)


def _random(seed):
    g = np.random.default_rng(seed)
    R = int(g.integers(1, 90))
    C = int(g.integers(2, 700))
    S = int(g.integers(1, 9))
    elev = np.radians(np.sort(g.uniform(-25, 12, R))[::-1])
    rng = g.uniform(3.0, 9.0, (R, C)).astype(np.float32)
    rng[g.random((R, C)) > g.uniform(0.4, 0.95)] = 0.0
    tuning = [(0, 0, 0), (64, 128, 64), (512, 256, 64), (2048, 512, 8), (16384, 512, 0)][
        int(g.integers(0, 5))]
    return rng, elev, 2 * math.pi / C, float(g.uniform(0.2, 1.2)), S, bool(g.integers(0, 2)), tuning


@pytest.mark.parametrize("seed", range(40))
def test_random_frames(flic, seed):
    rng, elev, az, delta, S, wrap, tuning = _random(seed)
    try:
        _check(flic, rng, elev, az, delta, S, wrap, tuning)
    except flic.FlicError as e:  # a strip layout the frame does not fit
        assert e.status == flic.FLIC_ERR_UNSUPPORTED
        _check(flic, rng, elev, az, delta, S, wrap)


@pytest.mark.parametrize("shape,S", [((4, 3), 4), ((5, 7), 6), ((2, 5), 8), ((3, 9), 2)])
def test_narrow_wrapping_frames(flic, shape, S):
    """A single strip narrower than S wraps onto itself (the narrow border path)."""
    g = np.random.default_rng(sum(shape) + S)
    rng = g.uniform(4.0, 5.0, shape).astype(np.float32)
    rng[g.random(shape) > 0.8] = 0.0
    elev = np.radians(np.linspace(5.0, -5.0, shape[0]))
    _check(flic, rng, elev, 2 * math.pi / shape[1], 0.9, S, True)


def test_with_ground_extraction(flic):
    f = synth.config_c2()
    _check(flic, f.range, f.sensor.elevation, f.sensor.az_step, f.delta, 3, True,
           ground=(math.radians(10.0), 1.7))


def test_batch_mixed(flic):
    """The c4 batch with every other frame's handle on the sparse map."""
    frames = synth.config_c4(48)
    hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                           f.delta, f.skip, lattice=bool(i % 2)) for i, f in enumerate(frames)]
    try:
        rs = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in frames]
        ls = [torch.empty(f.range.size, dtype=torch.int32, device=DEV) for f in frames]
        b = flic.flic_batch_create(len(frames))
        flic.flic_label_batch(b, flic.BatchArgs(hs, rs, ls))
        torch.cuda.synchronize()
        for i, (f, lab) in enumerate(zip(frames, ls)):
            want = oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip,
                                lattice=bool(i % 2))
            np.testing.assert_array_equal(lab.cpu().numpy(), want.reshape(-1), err_msg=str(i))
        b.close()
    finally:
        for h in hs:
            h.close()
