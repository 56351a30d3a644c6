"""GPU parity of ground extraction (§III-A) before labelling: flic_set_ground, then
flic_label / flic_label_batch / flic_edges, element by element against the oracle
(oracle.label_ground, oracle.edges on the readings with the ground removed)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2003_00575_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
TEN = math.radians(10.0)


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


def _gpu(flic, rng, elev, az, delta, skip, wrap, theta, height, tuning=None):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap)
    try:
        if tuning:
            flic.flic_set_tuning(h, *tuning)
        flic.flic_set_ground(h, theta, height)
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        lab = torch.full((R * C,), 12345, dtype=torch.int32, device=DEV)
        m = torch.zeros(R * C, dtype=torch.int16, device=DEV)
        flic.flic_label(h, r, lab)
        flic.flic_edges(h, r, m)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        return (lab.cpu().numpy().reshape(R, C),
                m.cpu().numpy().view(np.uint16).reshape(R, C))
    finally:
        h.close()


def _check(flic, rng, elev, az, delta, skip, wrap, theta, height, tuning=None):
    lab, edges = _gpu(flic, rng, elev, az, delta, skip, wrap, theta, height, tuning)
    want = oracle.label_ground(rng, elev, az, delta, skip, wrap, theta, height)
    np.testing.assert_array_equal(lab, want)
    g = oracle.ground(rng, elev, theta, height)
    cleared = np.where(g, np.float32(0), np.asarray(rng, np.float32))
    np.testing.assert_array_equal(edges, oracle.edges(cleared, elev, az, delta, skip, wrap))
    return g


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
@pytest.mark.parametrize("height", [0.0, 1.7])
def test_configs(flic, name, height):
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[name]()
    g = _check(flic, f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip, True,
               TEN, height)
    assert g.mean() > 0.05  # the scenes' ground plane is found


def _random(seed):
    g = np.random.default_rng(seed)
    R = int(g.integers(2, 70))
    C = int(g.integers(3, 500))
    S = int(g.integers(1, 7))
    elev = np.radians(np.sort(g.uniform(-30, 10, R))[::-1])
    # a ground plane under noise-free boxes and random clutter
    rng = np.zeros((R, C))
    for r in range(R):
        if elev[r] < -0.01:
            rng[r, :] = 1.7 / math.sin(-elev[r])
    clutter = g.random((R, C)) < 0.3
    rng[clutter] = g.uniform(1.0, 20.0, clutter.sum())
    rng[g.random((R, C)) < 0.1] = 0.0
    theta = math.radians(float(g.uniform(1.0, 35.0)))
    height = float(g.choice([0.0, 1.7, 0.5]))
    tuning = [(0, 0, 0), (64, 128, 64), (256, 256, 8), (2048, 512, 3)][int(g.integers(0, 4))]
    return (rng.astype(np.float32), elev, 2 * math.pi / C, float(g.uniform(0.2, 1.0)), S,
            bool(g.integers(0, 2)), theta, height, tuning)


@pytest.mark.parametrize("seed", range(24))
def test_random_frames(flic, seed):
    """Many strips (border merges test the ground at strip borders), wrap on and off."""
    rng, elev, az, delta, S, wrap, theta, height, tuning = _random(seed)
    _check(flic, rng, elev, az, delta, S, wrap, theta, height, tuning)


def test_off_and_single_row(flic):
    f = synth.config_c1()
    args = (f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip, True)
    lab0, _ = _gpu(flic, *args, 0.0, 0.0)
    np.testing.assert_array_equal(lab0, oracle.label(*args).reshape(lab0.shape))
    one = np.full((1, 40), 3.0, np.float32)
    lab1, _ = _gpu(flic, one, np.array([-0.2]), 2 * math.pi / 40, 0.5, 1, True, TEN, 0.0)
    assert (lab1 == 0).all()  # one row has no row above: nothing is ground


def test_batch_c4(flic):
    frames = synth.config_c4(64)
    hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                           f.delta, f.skip) for f in frames]
    try:
        for h in hs:
            flic.flic_set_ground(h, TEN, 1.7)
        rs = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in frames]
        ls = [torch.empty(f.range.size, dtype=torch.int32, device=DEV) for f in frames]
        b = flic.flic_batch_create(len(frames))
        flic.flic_label_batch(b, flic.BatchArgs(hs, rs, ls))
        torch.cuda.synchronize()
        for f, lab in zip(frames, ls):
            want = oracle.label_ground(f.range, f.sensor.elevation, f.sensor.az_step, f.delta,
                                       f.skip, True, TEN, 1.7)
            np.testing.assert_array_equal(lab.cpu().numpy(), want.reshape(-1))
        b.close()
    finally:
        for h in hs:
            h.close()
