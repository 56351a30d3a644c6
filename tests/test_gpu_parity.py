"""GPU parity: libflic (through the C ABI) against the CPU oracle, element by element.

Integer outputs (labels, edge bits, pixel indices) and the projected ranges must be
bit-exact; both sides evaluate the same fp32 expressions without contraction.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2003_00575_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


DEV = "cuda"


def gpu_label(flic, rng, elev, az, delta, skip, wrap=True, tuning=None):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap)
    try:
        if tuning:
            flic.flic_set_tuning(h, *tuning)
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        lab = torch.full((R * C,), 12345, dtype=torch.int32, device=DEV)
        flic.flic_label(h, r, lab)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        return lab.cpu().numpy().reshape(R, C)
    finally:
        h.close()


def gpu_edges(flic, rng, elev, az, delta, skip, wrap=True):
    R, C = rng.shape
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap)
    try:
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        m = torch.zeros(R * C, dtype=torch.int16, device=DEV)
        flic.flic_edges(h, r, m)
        torch.cuda.synchronize()
        return m.cpu().numpy().view(np.uint16).reshape(R, C)
    finally:
        h.close()


def frame_args(f):
    return f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip


CONFIGS = {
    "c1": synth.config_c1,
    "c2": synth.config_c2,
    "c3": lambda: synth.config_c3(with_xyz=True),
}


@pytest.fixture(scope="module")
def frames():
    return {k: v() for k, v in CONFIGS.items()}


# ---------------------------------------------------------------- tables and edges

@pytest.mark.parametrize("name", list(CONFIGS))
def test_tables_bit_exact(flic, frames, name):
    f = frames[name]
    s = f.sensor
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, f.delta, f.skip)
    kv, kh = flic.flic_get_tables(h)
    h.close()
    kv_o, kh_o = oracle.tables(s.elevation, s.az_step, f.skip)
    np.testing.assert_array_equal(kv, kv_o)
    np.testing.assert_array_equal(kh, kh_o)


@pytest.mark.parametrize("name", list(CONFIGS))
def test_edges_bit_exact(flic, frames, name):
    f = frames[name]
    got = gpu_edges(flic, *frame_args(f))
    want = oracle.edges(*frame_args(f))
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- labels, full configs

@pytest.mark.parametrize("name", list(CONFIGS))
def test_labels_bit_exact_full_frames(flic, frames, name):
    f = frames[name]
    got = gpu_label(flic, *frame_args(f))
    want = oracle.label(*frame_args(f))
    np.testing.assert_array_equal(got, want)


def test_hand_example_on_gpu(flic, golden_dir):
    import json
    import os
    g = json.load(open(os.path.join(golden_dir, "hand_3x4.json")))
    elev = np.radians(g["elevation_deg"])
    az = math.radians(g["az_step_deg"])
    rng = np.array(g["range"], np.float32)
    for case in g["cases"]:
        got = gpu_label(flic, rng, elev, az, case["delta"], case["skip"], wrap=case["wrap"])
        np.testing.assert_array_equal(got, np.array(case["labels"]), err_msg=str(case))


TUNINGS = [(0, 0, 0), (64, 128, 64), (256, 256, 4), (1024, 512, 8), (4096, 512, 4),
           (32768, 256, 4), (512, 128, 16), (8192, 512, 12), (2048, 256, 64)]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_labels_independent_of_launch_shape(flic, frames, tuning):
    f = frames["c2"]
    want = oracle.label(*frame_args(f))
    got = gpu_label(flic, *frame_args(f), tuning=tuning)
    np.testing.assert_array_equal(got, want)


# ---------------------------------------------------------------- random shapes, edge cases

def _random_frame(seed):
    g = np.random.default_rng(seed)
    R = int(g.integers(1, 80))
    C = int(g.integers(1, 400))
    S = int(g.integers(1, 9))
    wrap = bool(g.integers(0, 2))
    kind = int(g.integers(0, 3))
    if kind == 0:   # smooth surface with holes: long runs, big components
        base = 5 + 3 * np.sin(np.arange(C) / 17.0)[None, :] + 0.05 * np.arange(R)[:, None]
        rng = base + g.normal(0, 0.05, (R, C))
        rng[g.random((R, C)) < 0.15] = 0
    elif kind == 1:  # few distinct values: ties, invalid readings of every kind
        vals = np.array([0.0, 1.0, 1.2, 2.0, 2.1, 7.0, np.nan, np.inf, -3.0])
        rng = vals[g.integers(0, len(vals), (R, C))]
    else:            # noise: many small components
        rng = g.uniform(0.5, 30, (R, C))
        rng[g.random((R, C)) < 0.3] = 0
    elev = np.radians(np.linspace(10, -10, R)) if R > 1 else np.array([0.0])
    az = 2 * math.pi / C
    delta = float(np.float32(g.uniform(0.1, 1.5)))
    tuning = [(0, 0, 0), (64, 128, 64), (128, 256, 8), (1024, 512, 3)][int(g.integers(0, 4))]
    return rng.astype(np.float32), elev, az, delta, S, wrap, tuning


@pytest.mark.parametrize("seed", range(60))
def test_labels_random_shapes(flic, seed):
    rng, elev, az, delta, S, wrap, tuning = _random_frame(seed)
    want = oracle.label(rng, elev, az, delta, S, wrap=wrap)
    got = gpu_label(flic, rng, elev, az, delta, S, wrap=wrap, tuning=tuning)
    np.testing.assert_array_equal(got, want)
    gotm = gpu_edges(flic, rng, elev, az, delta, S, wrap=wrap)
    np.testing.assert_array_equal(gotm, oracle.edges(rng, elev, az, delta, S, wrap=wrap))


DEGENERATE = {
    "1x1": np.array([[3.0]]),
    "1x1_invalid": np.array([[0.0]]),
    "row": np.full((1, 257), 4.0),
    "column": np.full((300, 1), 4.0),
    "all_invalid": np.zeros((16, 200)),
    "all_nan": np.full((8, 64), np.nan),
    "one_component": np.full((64, 512), 10.0),
    "checkerboard": np.indices((40, 96)).sum(0) % 2 * 5.0,
    "narrow_cols_lt_2S": np.full((20, 5), 2.0),
    "rows_le_S": np.full((3, 120), 2.0),
    "stripes": np.tile(np.array([1.0, 1.0, 0.0, 50.0]), (12, 40)),
}


@pytest.mark.parametrize("name", list(DEGENERATE))
@pytest.mark.parametrize("skip,wrap,tuning", [(1, True, (0, 0, 0)), (5, True, (64, 128, 64)),
                                              (8, False, (128, 256, 4)), (3, False, (0, 0, 0))])
def test_labels_degenerate(flic, name, skip, wrap, tuning):
    rng = DEGENERATE[name].astype(np.float32)
    R, C = rng.shape
    elev = np.radians(np.linspace(5, -5, R)) if R > 1 else np.array([0.0])
    az = 2 * math.pi / C
    want = oracle.label(rng, elev, az, 0.5, skip, wrap=wrap)
    got = gpu_label(flic, rng, elev, az, 0.5, skip, wrap=wrap, tuning=tuning)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("shape", [(128, 4096), (512, 1024), (16, 32768), (256, 8192)])
def test_largest_frames(flic, shape):
    """Large frames up to the documented pixel limit (2^21), split over up to 64 strips."""
    R, C = shape
    g = np.random.default_rng(R)
    base = 20 + 5 * np.sin(np.arange(C) / 50.0)[None, :] + 0.01 * np.arange(R)[:, None]
    rng = (base + g.normal(0, 0.02, (R, C))).astype(np.float32)
    rng[g.random((R, C)) < 0.1] = 0
    elev = np.radians(np.linspace(20, -20, R))
    az = 2 * math.pi / C
    want = oracle.label(rng, elev, az, 0.5, 3)
    got = gpu_label(flic, rng, elev, az, 0.5, 3)
    np.testing.assert_array_equal(got, want)


def test_oversized_frame_rejected(flic):
    with pytest.raises(flic.FlicError) as e:
        flic.flic_create(512, 8192, np.zeros(512), 2 * math.pi / 8192, 0.5, 1)
    assert e.value.status == flic.FLIC_ERR_INVALID


def test_timeout_reported_not_hung(flic, frames):
    """An iteration budget of 1 makes the union loops give up: the kernel returns, the
    status word says so, and the handle keeps working after a reset."""
    f = frames["c2"]
    s = f.sensor
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, f.delta, f.skip)
    try:
        r = torch.from_numpy(f.range).to(DEV)
        lab = torch.empty(s.rows * s.cols, dtype=torch.int32, device=DEV)
        flic.flic_debug_set_iter_limit(h, 1)
        flic.flic_label(h, r, lab)
        assert flic.flic_device_status(h, clear=True) == flic.FLIC_ERR_TIMEOUT
        flic.flic_debug_set_iter_limit(h, 0)
        flic.flic_label(h, r, lab)
        assert flic.flic_device_status(h) == flic.FLIC_OK
        np.testing.assert_array_equal(lab.cpu().numpy().reshape(s.rows, s.cols),
                                      oracle.label(*frame_args(f)))
    finally:
        h.close()


# ---------------------------------------------------------------- projection and scatter

def gpu_project(flic, f, xyz):
    s = f.sensor
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, f.delta, f.skip)
    try:
        xt = torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).to(DEV)
        rimg = torch.empty(s.rows * s.cols, dtype=torch.float32, device=DEV)
        pix = torch.empty(xyz.shape[0], dtype=torch.int32, device=DEV)
        flic.flic_project(h, xt, rimg, pix)
        lab = torch.empty(s.rows * s.cols, dtype=torch.int32, device=DEV)
        flic.flic_label(h, rimg, lab)
        plab = torch.empty_like(pix)
        flic.flic_scatter(h, lab, pix, plab)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        return (rimg.cpu().numpy().reshape(s.rows, s.cols), pix.cpu().numpy(),
                lab.cpu().numpy().reshape(s.rows, s.cols), plab.cpu().numpy())
    finally:
        h.close()


def _check_projection(flic, f, xyz):
    s = f.sensor
    rimg, pix, lab, plab = gpu_project(flic, f, xyz)
    r_o, pix_o, _ = oracle.project(xyz, s.rows, s.cols, s.elevation, s.az_step)
    np.testing.assert_array_equal(pix, pix_o)
    np.testing.assert_array_equal(rimg.view(np.uint32), r_o.view(np.uint32))
    lab_o = oracle.label(r_o, s.elevation, s.az_step, f.delta, f.skip)
    np.testing.assert_array_equal(lab, lab_o)
    np.testing.assert_array_equal(plab, oracle.scatter(lab_o, pix_o))


def test_projection_c3_one_point_per_pixel(flic, frames):
    f = frames["c3"]
    _check_projection(flic, f, f.xyz)


@pytest.mark.parametrize("seed,shape", [(1000, 0), (1001, 1), (1002, 2), (1003, 3)])
def test_projection_clouds_with_collisions(flic, seed, shape):
    s = synth.c5_sensors()[shape]
    f = synth.c5_frame(s, seed, as_cloud=True)
    _check_projection(flic, f, f.xyz)


def test_projection_random_directions(flic):
    s = synth.make_sensor(64, 2048, -22.5, 22.5)
    g = np.random.default_rng(3)
    n = 300_000
    d = g.uniform(0.3, 150, n)
    az = g.uniform(0, 2 * math.pi, n)
    el = g.uniform(math.radians(-30), math.radians(30), n)
    xyz = np.stack([d * np.cos(el) * np.cos(az), d * np.cos(el) * np.sin(az), d * np.sin(el)],
                   1).astype(np.float32)
    xyz[::97] = 0.0
    xyz[5::101, 0] = np.nan
    f = synth.Frame(s, np.zeros((64, 2048), np.float32), 0.5, 2, None)
    _check_projection(flic, f, xyz)


def test_projection_empty_cloud(flic):
    s = synth.make_sensor(16, 1800, -15, 15)
    f = synth.Frame(s, np.zeros((16, 1800), np.float32), 0.5, 1, None)
    rimg, pix, lab, plab = gpu_project(flic, f, np.zeros((0, 3), np.float32))
    assert pix.shape == (0,) and np.all(rimg == 0) and np.all(lab == -1)


# ---------------------------------------------------------------- batch

def _run_batch(flic, fr, tuning=None, repeat=1):
    handles = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation,
                                f.sensor.az_step, f.delta, f.skip) for f in fr]
    ranges = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in fr]
    labels = [torch.full((f.range.size,), 777, dtype=torch.int32, device=DEV) for f in fr]
    b = flic.flic_batch_create(len(fr))
    try:
        if tuning:
            flic.flic_batch_set_tuning(b, *tuning)
        args = flic.BatchArgs(handles, ranges, labels)
        for _ in range(repeat):
            flic.flic_label_batch(b, args)
        torch.cuda.synchronize()
        st = [flic.flic_device_status(h) for h in handles]
        assert all(x == flic.FLIC_OK for x in st), st
        return [l.cpu().numpy().reshape(f.range.shape) for l, f in zip(labels, fr)], \
            flic.flic_batch_last_plan(b)
    finally:
        b.close()
        for h in handles:
            h.close()


@pytest.fixture(scope="module")
def c4_frames():
    return synth.config_c4(256)


@pytest.fixture(scope="module")
def c4_oracle(c4_frames):
    return [oracle.label(*frame_args(f)) for f in c4_frames]


def test_batch_full_c4_matches_oracle(flic, c4_frames, c4_oracle):
    got, plan = _run_batch(flic, c4_frames, repeat=2)
    assert plan["frames"] == 256
    bad = [(i, c4_frames[i].name, int((g != w).sum())) for i, (g, w) in
           enumerate(zip(got, c4_oracle)) if not np.array_equal(g, w)]
    assert not bad, (plan, bad[:20], len(bad))


@pytest.mark.parametrize("tuning", [(4096, 256, 64, 0), (16384, 512, 16, 1), (32768, 512, 8, 0),
                                    (2048, 128, 64, 2), (8192, 256, 64, 1)])
def test_batch_shapes_and_tunings(flic, c4_frames, c4_oracle, tuning):
    idx = list(range(0, 256, 7))
    got, _ = _run_batch(flic, [c4_frames[i] for i in idx], tuning=tuning)
    for g, i in zip(got, idx):
        np.testing.assert_array_equal(g, c4_oracle[i], err_msg=c4_frames[i].name)


def test_batch_equals_single_frame_calls(flic, c4_frames):
    fr = c4_frames[:24]
    got, _ = _run_batch(flic, fr)
    for g, f in zip(got, fr):
        np.testing.assert_array_equal(g, gpu_label(flic, *frame_args(f)))


def test_batch_capacity_error(flic):
    b = flic.flic_batch_create(1)
    try:
        f = synth.config_c1()
        h = flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                             f.delta, f.skip)
        r = torch.from_numpy(f.range.reshape(-1)).to(DEV)
        l1 = torch.empty(f.range.size, dtype=torch.int32, device=DEV)
        l2 = torch.empty_like(l1)
        args = flic.BatchArgs([h, h], [r, r], [l1, l2])
        with pytest.raises(flic.FlicError) as e:
            flic.flic_label_batch(b, args)
        assert e.value.status == flic.FLIC_ERR_BUSY
        h.close()
    finally:
        b.close()
