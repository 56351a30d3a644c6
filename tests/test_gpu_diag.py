"""GPU parity of the diagonal Map Connections (FLIC_FLAG_DIAGONAL, §III-B-2): the diagonal
constants and the labels against the oracle, element by element — full c1-c3 frames,
random shapes over launch shapes that force many strip borders and the narrow single-strip
case, degenerate frames, the exact-ray variant and the batch."""
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


def _label(flic, rng, elev, az, delta, skip, wrap=True, tuning=None, exact_ray=False):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap, exact_ray=exact_ray,
                         diagonal=True)
    try:
        if tuning:
            flic.flic_set_tuning(h, *tuning)
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        lab = torch.full((R * C,), 4242, dtype=torch.int32, device=DEV)
        flic.flic_label(h, r, lab)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        return flic.flic_get_diag_table(h), lab.cpu().numpy().reshape(R, C)
    finally:
        h.close()


CONFIGS = {"c1": synth.config_c1, "c2": synth.config_c2,
           "c3": lambda: synth.config_c3(with_xyz=False)}


@pytest.mark.parametrize("name", list(CONFIGS))
@pytest.mark.parametrize("tuning", [None, (512, 256, 64)])
def test_configs(flic, name, tuning):
    f = CONFIGS[name]()
    s = f.sensor
    kd, got = _label(flic, f.range, s.elevation, s.az_step, f.delta, f.skip, tuning=tuning)
    np.testing.assert_array_equal(kd, oracle.tables_diag(s.elevation, s.az_step, f.skip))
    want = oracle.label(f.range, s.elevation, s.az_step, f.delta, f.skip, diagonal=True)
    np.testing.assert_array_equal(got, want)
    # the diagonals change the partition of these frames
    assert not np.array_equal(want, oracle.label(f.range, s.elevation, s.az_step, f.delta,
                                                 f.skip))


def _random_frame(seed):
    g = np.random.default_rng(7000 + seed)
    R, C, S = int(g.integers(1, 70)), int(g.integers(1, 300)), int(g.integers(1, 9))
    kind = int(g.integers(0, 3))
    if kind == 0:
        base = 5 + 3 * np.sin(np.arange(C) / 11.0)[None, :] + 0.05 * np.arange(R)[:, None]
        rng = base + g.normal(0, 0.06, (R, C))
        rng[g.random((R, C)) < 0.2] = 0
    elif kind == 1:
        vals = np.array([0.0, 1.0, 1.2, 2.0, 2.1, 7.0, np.nan, np.inf, -3.0])
        rng = vals[g.integers(0, len(vals), (R, C))]
    else:
        rng = g.uniform(0.5, 30, (R, C))
        rng[g.random((R, C)) < 0.3] = 0
    elev = np.radians(np.linspace(10, -10, R)) if R > 1 else np.array([0.0])
    tuning = [(0, 0, 0), (64, 128, 64), (128, 256, 8), (1024, 512, 3)][int(g.integers(0, 4))]
    return (rng.astype(np.float32), elev, 2 * math.pi / C, float(np.float32(g.uniform(0.1, 1.5))),
            S, bool(g.integers(0, 2)), tuning)


@pytest.mark.parametrize("seed", range(40))
def test_random_shapes(flic, seed):
    rng, elev, az, delta, S, wrap, tuning = _random_frame(seed)
    _, got = _label(flic, rng, elev, az, delta, S, wrap=wrap, tuning=tuning)
    want = oracle.label(rng, elev, az, delta, S, wrap=wrap, diagonal=True)
    np.testing.assert_array_equal(got, want)


DEGENERATE = {
    "row": np.full((1, 257), 4.0),
    "column": np.full((300, 1), 4.0),
    "narrow_cols_lt_S": np.full((20, 5), 2.0),
    "checkerboard": np.indices((40, 96)).sum(0) % 2 * 5.0,
    "stripes": np.tile(np.array([1.0, 0.0, 1.0, 50.0]), (12, 40)),
    "diag_only": np.eye(48, 64)[::-1] * 3.0 + np.eye(48, 64) * 3.0,
}


@pytest.mark.parametrize("name", list(DEGENERATE))
@pytest.mark.parametrize("skip,wrap,tuning", [(1, True, (0, 0, 0)), (5, True, (64, 128, 64)),
                                              (8, False, (128, 256, 4)), (3, False, (0, 0, 0))])
def test_degenerate(flic, name, skip, wrap, tuning):
    rng = DEGENERATE[name].astype(np.float32)
    R, C = rng.shape
    elev = np.radians(np.linspace(5, -5, R)) if R > 1 else np.array([0.0])
    az = 2 * math.pi / C
    _, got = _label(flic, rng, elev, az, 0.5, skip, wrap=wrap, tuning=tuning)
    np.testing.assert_array_equal(got, oracle.label(rng, elev, az, 0.5, skip, wrap=wrap,
                                                    diagonal=True))


def test_with_exact_ray(flic):
    f = synth.config_c2()
    s = f.sensor
    _, got = _label(flic, f.range, s.elevation, s.az_step, f.delta, f.skip, exact_ray=True)
    np.testing.assert_array_equal(got, oracle.label(f.range, s.elevation, s.az_step, f.delta,
                                                    f.skip, exact_ray=True, diagonal=True))


def test_batch_mixes_diagonal_and_plain_frames(flic):
    fr = synth.config_c4(24)
    hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                           f.delta, f.skip, diagonal=(i % 2 == 0)) for i, f in enumerate(fr)]
    rg = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in fr]
    lb = [torch.full((f.range.size,), 99, dtype=torch.int32, device=DEV) for f in fr]
    b = flic.flic_batch_create(len(fr))
    try:
        flic.flic_label_batch(b, flic.BatchArgs(hs, rg, lb))
        torch.cuda.synchronize()
        assert all(flic.flic_device_status(h) == flic.FLIC_OK for h in hs)
        for i, (f, l) in enumerate(zip(fr, lb)):
            s = f.sensor
            want = oracle.label(f.range, s.elevation, s.az_step, f.delta, f.skip,
                                diagonal=(i % 2 == 0))
            np.testing.assert_array_equal(l.cpu().numpy().reshape(f.range.shape), want,
                                          err_msg=f.name)
    finally:
        b.close()
        for h in hs:
            h.close()
