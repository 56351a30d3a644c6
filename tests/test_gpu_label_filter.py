"""GPU parity of flic_label_filter_batch: labelling and the cluster-candidate filter
(§III-B) in one call, the component sizes counted inside the labelling kernel (strip-local
runs in the strip pass, hooked roots added after the border merges).  Element by element
against oracle.filter_relabel on the oracle's labels, over the c4 batch, ragged shapes,
many-strip tunings, wrap and no wrap, the sparse and diagonal Map Connections and ground
extraction; and the plain labelling calls on the same batch object stay unchanged."""
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


def _fused(flic, b, hs, ranges, m, fill=777):
    """flic_label_filter_batch over host frames; returns (labels list, N list)."""
    rs = [torch.from_numpy(np.ascontiguousarray(x, np.float32).reshape(-1)).to(DEV)
          for x in ranges]
    ls = [torch.full((x.size,), fill, dtype=torch.int32, device=DEV) for x in ranges]
    num = torch.full((len(hs),), -7, dtype=torch.int32, device=DEV)
    flic.flic_label_filter_batch(b, flic.BatchArgs(hs, rs, ls), m, num)
    torch.cuda.synchronize()
    for h in hs:
        assert flic.flic_device_status(h) == flic.FLIC_OK
    return [x.cpu().numpy() for x in ls], [int(v) for v in num.cpu().numpy()]


def _check(got, nums, wants):
    for i, ((g, n), (w, wn)) in enumerate(zip(zip(got, nums), wants)):
        assert np.array_equal(g, w.reshape(-1)), (i, int((g != w.reshape(-1)).sum()))
        assert n == wn, (i, n, wn)


@pytest.fixture(scope="module")
def c4():
    frames = synth.config_c4(256)
    labels = [oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
              for f in frames]
    return frames, labels


def _handles(flic, frames, **kw):
    return [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation,
                             f.sensor.az_step, f.delta, f.skip, **kw) for f in frames]


@pytest.mark.parametrize("m", [100, 1])
def test_c4_batch(flic, c4, m):
    """The full c4 batch in one call, twice (the second replays the labelling graph)."""
    frames, labels = c4
    hs = _handles(flic, frames)
    b = flic.flic_batch_create(len(frames))
    try:
        wants = [oracle.filter_relabel(l, m) for l in labels]
        for _ in range(2):
            got, nums = _fused(flic, b, hs, [f.range for f in frames], m)
            _check(got, nums, wants)
    finally:
        b.close()
        for h in hs:
            h.close()


@pytest.mark.parametrize("tuning", [(2048, 128, 64, 2), (4096, 256, 64, 0),
                                    (32768, 512, 8, 0)])
def test_c4_many_strips(flic, c4, tuning):
    """Small strips: many borders per frame, so most strip-local roots are hooked and their
    counts move to other strips' roots."""
    frames, labels = c4
    idx = list(range(3, 256, 11))
    hs = _handles(flic, [frames[i] for i in idx])
    b = flic.flic_batch_create(len(idx))
    try:
        flic.flic_batch_set_tuning(b, *tuning)
        got, nums = _fused(flic, b, hs, [frames[i].range for i in idx], 30)
        _check(got, nums, [oracle.filter_relabel(labels[i], 30) for i in idx])
    finally:
        b.close()
        for h in hs:
            h.close()


def _noise(R, C, seed, p=0.75):
    g = np.random.default_rng(seed)
    rng = g.uniform(4.0, 6.0, (R, C)).astype(np.float32)
    rng[g.random((R, C)) > p] = 0.0
    elev = np.radians(np.linspace(15.0, -15.0, R)) if R > 1 else np.array([0.0])
    return rng, elev, 2 * np.pi / C, float(np.float32(g.uniform(0.2, 0.6))), int(g.integers(1, 7))


@pytest.mark.parametrize("wrap", [True, False])
def test_ragged_shapes(flic, wrap):
    """Frames smaller than a relabel tile, ragged rows and tiles, odd widths (scalar label
    stores), one column, one row; one batch, several min sizes."""
    shapes = [(1, 1), (1, 7), (3, 3), (5, 819), (64, 64), (7, 4097), (33, 1000), (16, 1800),
              (2, 3001), (40, 33), (128, 2048), (9, 1)]
    frames = [_noise(R, C, 13 * R + C + wrap) for R, C in shapes]
    hs = [flic.flic_create(r.shape[0], r.shape[1], e, a, d, s, wrap=wrap)
          for r, e, a, d, s in frames]
    b = flic.flic_batch_create(len(frames))
    try:
        refs = [oracle.label(r, e, a, d, s, wrap) for r, e, a, d, s in frames]
        for m in (0, 2, 9, 40):
            got, nums = _fused(flic, b, hs, [f[0] for f in frames], m)
            _check(got, nums, [oracle.filter_relabel(l, m) for l in refs])
    finally:
        b.close()
        for h in hs:
            h.close()


def test_one_component_and_no_measurement(flic):
    """A frame that is one component of every pixel (its root's count is the whole frame,
    summed over every strip), next to a frame with no measurement at all."""
    R, C = 64, 2048
    elev = np.radians(np.linspace(10.0, -10.0, R))
    full = np.full((R, C), 5.0, np.float32)
    empty = np.zeros((R, C), np.float32)
    hs = [flic.flic_create(R, C, elev, 2 * np.pi / C, 50.0, 2) for _ in range(2)]
    b = flic.flic_batch_create(2)
    try:
        flic.flic_batch_set_tuning(b, 2048, 256, 64, 0)
        for m in (R * C, R * C + 1):
            got, nums = _fused(flic, b, hs, [full, empty], m)
            keep = m <= R * C
            assert np.all(got[0] == (0 if keep else -1)) and nums[0] == int(keep)
            assert np.all(got[1] == -1) and nums[1] == 0
    finally:
        b.close()
        for h in hs:
            h.close()


@pytest.mark.parametrize("variant", ["lattice", "diagonal", "ground"])
def test_map_connection_variants(flic, variant):
    """The sparse and diagonal Map Connections and ground extraction: the counts follow the
    variant's components."""
    s = synth.c5_sensors()[2]
    frames = [synth.c5_frame(s, 900 + i, as_cloud=False) for i in range(6)]
    kw = {"lattice": {"lattice": True}, "diagonal": {"diagonal": True}}.get(variant, {})
    hs = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3, **kw)
          for _ in frames]
    theta, height = np.radians(10.0), 1.7
    if variant == "ground":
        for h in hs:
            flic.flic_set_ground(h, theta, height)
    b = flic.flic_batch_create(len(frames))
    try:
        flic.flic_batch_set_tuning(b, 4096, 256, 64, 0)
        if variant == "ground":
            refs = [oracle.label_ground(f.range, s.elevation, s.az_step, 0.5, 3, True, theta,
                                        height) for f in frames]
        else:
            refs = [oracle.label(f.range, s.elevation, s.az_step, 0.5, 3, **kw) for f in frames]
        got, nums = _fused(flic, b, hs, [f.range for f in frames], 20)
        _check(got, nums, [oracle.filter_relabel(l, 20) for l in refs])
    finally:
        b.close()
        for h in hs:
            h.close()


def test_plain_calls_on_the_same_batch(flic, c4):
    """Fused, plain labelling, fused, separate label + filter on one batch object: the plain
    call gets component minima (no counting), every result is exact."""
    frames, labels = c4
    fr = frames[:32]
    hs = _handles(flic, fr)
    rs = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in fr]
    ls = [torch.empty(f.range.size, dtype=torch.int32, device=DEV) for f in fr]
    args = flic.BatchArgs(hs, rs, ls)
    num = torch.zeros(len(fr), dtype=torch.int32, device=DEV)
    b = flic.flic_batch_create(len(fr))
    wants = [oracle.filter_relabel(l, 100) for l in labels[:32]]
    try:
        for step in ("fused", "plain", "fused", "separate", "fused"):
            if step == "fused":
                flic.flic_label_filter_batch(b, args, 100, num)
            else:
                flic.flic_label_batch(b, args)
                if step == "separate":
                    flic.flic_filter_relabel_batch(b, args, 100, num)
            torch.cuda.synchronize()
            for i in range(len(fr)):
                got = ls[i].cpu().numpy()
                if step == "plain":
                    assert np.array_equal(got, labels[i].reshape(-1)), (step, i)
                else:
                    assert np.array_equal(got, wants[i][0].reshape(-1)), (step, i)
                    assert int(num[i].item()) == wants[i][1], (step, i)
        assert all(flic.flic_device_status(h) == flic.FLIC_OK for h in hs)
    finally:
        b.close()
        for h in hs:
            h.close()


def test_changing_frame_sets_regrow_the_scratch(flic):
    """Consecutive fused calls on different frame sets (fewer tiles, more, fewer again):
    the root bitmask is cleared each call and the counts are exact every time."""
    b = flic.flic_batch_create(48)
    sets = [synth.config_c4(12, 300), synth.config_c4(3, 400), synth.config_c4(40, 500),
            synth.config_c4(5, 600), synth.config_c4(12, 300)]
    try:
        for k, frames in enumerate(sets):
            hs = _handles(flic, frames)
            try:
                m = (100, 1, 30, 100, 7)[k]
                got, nums = _fused(flic, b, hs, [f.range for f in frames], m)
                refs = [oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta,
                                     f.skip) for f in frames]
                _check(got, nums, [oracle.filter_relabel(l, m) for l in refs])
            finally:
                for h in hs:
                    h.close()
    finally:
        b.close()


def test_hooked_rows_only_low_in_the_frame(flic):
    """Components that cross strip borders only low in the frame (a full bottom row, a
    two-row band in the middle) under components that stay inside one strip: the flatten
    of each strip starts at its topmost hooked root, and the labels above it (plain and
    fused calls, with and without wrap) still equal the oracle's."""
    R, C = 16, 512
    elev = np.radians(np.linspace(10.0, -10.0, R))
    rng = np.zeros((R, C), np.float32)
    rng[0:4, 10:21] = 5.0       # inside the first strip
    rng[5:9, 300:310] = 5.0     # inside a middle strip
    rng[6:8, 100:200] = 5.0     # crosses the border between the first two strips
    rng[15, :] = 5.0            # the bottom row crosses every border
    for wrap in (True, False):
        hs = [flic.flic_create(R, C, elev, 2 * np.pi / C, 50.0, 1, wrap=wrap)]
        b = flic.flic_batch_create(1)
        try:
            flic.flic_batch_set_tuning(b, 2048, 128, 64, 0)  # 128-column strips
            ref = oracle.label(rng, elev, 2 * np.pi / C, 50.0, 1, wrap)
            r = torch.from_numpy(rng.reshape(-1)).to(DEV)
            lab = torch.full((R * C,), 777, dtype=torch.int32, device=DEV)
            flic.flic_label_batch(b, flic.BatchArgs(hs, [r], [lab]))
            torch.cuda.synchronize()
            assert flic.flic_batch_last_plan(b)["strips"] == 4
            assert np.array_equal(lab.cpu().numpy(), ref.reshape(-1)), wrap
            got, nums = _fused(flic, b, hs, [rng], 1)
            _check(got, nums, [oracle.filter_relabel(ref, 1)])
        finally:
            b.close()
            for h in hs:
                h.close()
