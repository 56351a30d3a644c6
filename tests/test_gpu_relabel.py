"""GPU parity of the cluster-candidate filter and compact numbering (§III-B) against the
oracle, element by element: flic_filter_relabel and flic_filter_relabel_batch on labels
produced by libflic, compared with oracle.filter_relabel on the oracle's own labels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2003_00575_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda"
SIZES = (0, 1, 2, 3, 10, 100, 1000, 1 << 30)


@pytest.fixture(scope="module")
def flic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_00575_gb300 import flic as _flic
    return _flic


def _check_frame(flic, rng, elev, az, delta, skip, wrap=True, sizes=SIZES):
    R, C = rng.shape
    ref_labels = oracle.label(rng, elev, az, delta, skip, wrap).reshape(R, C)
    h = flic.flic_create(R, C, elev, az, delta, skip, wrap=wrap)
    try:
        r = torch.from_numpy(np.ascontiguousarray(rng, np.float32)).to(DEV)
        base = torch.empty(R * C, dtype=torch.int32, device=DEV)
        flic.flic_label(h, r, base)
        num = torch.full((1,), -7, dtype=torch.int32, device=DEV)
        for m in sizes:
            lab = base.clone()
            flic.flic_filter_relabel(h, lab, m, num)
            torch.cuda.synchronize()
            assert flic.flic_device_status(h) == flic.FLIC_OK
            want, n = oracle.filter_relabel(ref_labels, m)
            got = lab.cpu().numpy().reshape(R, C)
            assert np.array_equal(got, want), (R, C, skip, m)
            assert int(num.item()) == n, (R, C, skip, m)
    finally:
        h.close()


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_configs(flic, name):
    f = {"c1": synth.config_c1, "c2": synth.config_c2,
         "c3": lambda: synth.config_c3(with_xyz=False)}[name]()
    _check_frame(flic, f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)


def _noise_frame(R, C, seed, p=0.7):
    g = np.random.default_rng(seed)
    rng = g.uniform(4.0, 6.0, (R, C)).astype(np.float32)
    rng[g.random((R, C)) > p] = 0.0
    elev = np.radians(np.linspace(15.0, -15.0, R)) if R > 1 else np.array([0.0])
    return rng, elev, 2 * np.pi / C, float(g.uniform(0.1, 0.6)), int(g.integers(1, 6))


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (3, 3), (5, 819), (64, 64), (7, 4097),
                                   (33, 1000), (16, 1800), (128, 2048)])
def test_shapes(flic, shape):
    """Tiles of 4096 pixels: frames smaller than one tile, ragged last tiles, many tiles."""
    R, C = shape
    rng, elev, az, delta, skip = _noise_frame(R, C, 7 * R + C)
    _check_frame(flic, rng, elev, az, delta, skip, sizes=(0, 1, 2, 5, 50))


def test_largest_frame(flic):
    """2^21 pixels: 512 tiles, the most one frame can have."""
    rng, elev, az, delta, skip = _noise_frame(512, 4096, 11, p=0.8)
    _check_frame(flic, rng, elev, az, delta, 1, sizes=(1, 100))


def test_all_invalid_and_one_component(flic):
    R, C = 9, 700
    elev = np.radians(np.linspace(10.0, -10.0, R))
    _check_frame(flic, np.zeros((R, C), np.float32), elev, 2 * np.pi / C, 0.5, 2)
    _check_frame(flic, np.full((R, C), 5.0, np.float32), elev, 2 * np.pi / C, 50.0, 2,
                 sizes=(0, R * C, R * C + 1))


def test_batch_c4(flic):
    """The c4 batch: labelled in one persistent launch, filtered in one set of launches with
    the paper's minimum of 100 points; every frame equals the oracle."""
    frames = synth.config_c4(256)
    hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                           f.delta, f.skip) for f in frames]
    try:
        rs = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in frames]
        ls = [torch.empty(f.range.size, dtype=torch.int32, device=DEV) for f in frames]
        b = flic.flic_batch_create(len(frames))
        args = flic.BatchArgs(hs, rs, ls)
        num = torch.full((len(frames),), -7, dtype=torch.int32, device=DEV)
        for rep in range(2):  # the second call reuses the batch's scratch
            flic.flic_label_batch(b, args)
            flic.flic_filter_relabel_batch(b, args, 100, num)
            torch.cuda.synchronize()
            nums = num.cpu().numpy()
            for i in (0, 1, 77, 128, 200, 255) if rep else range(len(frames)):
                f = frames[i]
                ref = oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
                want, n = oracle.filter_relabel(ref, 100)
                assert np.array_equal(ls[i].cpu().numpy(), want.reshape(-1)), (rep, i)
                assert nums[i] == n, (rep, i)
        b.close()
        for h in hs:
            assert flic.flic_device_status(h) == flic.FLIC_OK
    finally:
        for h in hs:
            h.close()


def test_batch_shares_a_handle(flic):
    """The same handle for several frames of one batch: the scratch is the batch's."""
    f = synth.config_c1()
    R, C = f.sensor.rows, f.sensor.cols
    h = flic.flic_create(R, C, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
    try:
        ranges = [f.range, np.roll(f.range, 37, axis=1), np.flip(f.range, axis=0).copy()]
        rs = [torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(DEV) for x in ranges]
        ls = [torch.empty(R * C, dtype=torch.int32, device=DEV) for _ in ranges]
        b = flic.flic_batch_create(3)
        args = flic.BatchArgs([h, h, h], rs, ls)
        flic.flic_label_batch(b, args)
        flic.flic_filter_relabel_batch(b, args, 5)
        torch.cuda.synchronize()
        for x, lab in zip(ranges, ls):
            ref = oracle.label(np.ascontiguousarray(x), f.sensor.elevation, f.sensor.az_step,
                               f.delta, f.skip)
            assert np.array_equal(lab.cpu().numpy(), oracle.filter_relabel(ref, 5)[0].reshape(-1))
        b.close()
    finally:
        h.close()


def test_out_of_frame_labels_are_reported(flic):
    """Values outside the frame are never used as an index: left in place, reported."""
    R, C = 4, 50
    elev = np.radians(np.linspace(5.0, -5.0, R))
    h = flic.flic_create(R, C, elev, 2 * np.pi / C, 0.5, 1)
    try:
        lab = torch.arange(R * C, dtype=torch.int32, device=DEV)  # every pixel its own root
        lab[3] = R * C + 5
        lab[10] = 1 << 30
        flic.flic_filter_relabel(h, lab, 1)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_ERR_INVALID
        got = lab.cpu().numpy()
        assert got[3] == R * C + 5 and got[10] == 1 << 30
        assert flic.flic_device_status(h) == flic.FLIC_OK  # cleared
    finally:
        h.close()


def _labelled(flic, frames):
    hs = [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                           f.delta, f.skip) for f in frames]
    ls = []
    for f, h in zip(frames, hs):
        r = torch.from_numpy(f.range.reshape(-1)).to(DEV)
        lab = torch.empty(f.range.size, dtype=torch.int32, device=DEV)
        flic.flic_label(h, r, lab)
        ls.append(lab)
    torch.cuda.synchronize()
    return hs, ls


def _want(f, m):
    ref = oracle.label(f.range, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
    return oracle.filter_relabel(ref, m)


def test_batch_scratch_across_changing_frame_sets(flic):
    """One batch object, consecutive calls on different frame sets (fewer tiles, then more,
    which regrows the scratch, then fewer again): the counts left at the previous call's
    roots are reset, every call equals the oracle."""
    b = flic.flic_batch_create(64)
    sets = [synth.config_c4(12, 300), synth.config_c4(3, 400), synth.config_c4(40, 500),
            synth.config_c4(5, 600), synth.config_c4(12, 300)]
    try:
        for k, frames in enumerate(sets):
            hs, ls = _labelled(flic, frames)
            try:
                num = torch.full((len(frames),), -7, dtype=torch.int32, device=DEV)
                m = (100, 1, 30, 100, 7)[k]
                flic.flic_filter_relabel_batch(b, _LabelArgs(flic, hs, ls), m, num)
                torch.cuda.synchronize()
                for i, f in enumerate(frames):
                    want, n = _want(f, m)
                    assert np.array_equal(ls[i].cpu().numpy(), want.reshape(-1)), (k, i)
                    assert int(num[i].item()) == n, (k, i)
                assert all(flic.flic_device_status(h) == flic.FLIC_OK for h in hs)
            finally:
                for h in hs:
                    h.close()
    finally:
        b.close()


class _LabelArgs:
    """BatchArgs for flic_filter_relabel_batch, which reads only the handles and labels."""

    def __init__(self, flic, hs, ls):
        import ctypes
        n = len(hs)
        self.n = n
        self.hs = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
        self.rs = None
        self.ls = (ctypes.c_void_p * n)(*[x.data_ptr() for x in ls])
        self._keep = (hs, ls)


def test_single_handle_consecutive_calls_and_stray_labels(flic):
    """One handle, one frame shape: different frames' labels one after another, and in
    between a call on labels that point at pixels which are not roots (unspecified ids):
    the calls after it are still exact."""
    s = synth.c5_sensors()[2]
    frames = [synth.c5_frame(s, 700 + i, as_cloud=False) for i in range(4)]
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3)
    try:
        num = torch.full((1,), -7, dtype=torch.int32, device=DEV)
        for k, f in enumerate(frames):
            r = torch.from_numpy(f.range.reshape(-1)).to(DEV)
            lab = torch.empty(f.range.size, dtype=torch.int32, device=DEV)
            flic.flic_label(h, r, lab)
            if k == 2:  # stray labels: every valid pixel points at its right-hand neighbour
                stray = torch.where(lab >= 0, (torch.arange(lab.numel(), device=DEV) + 1)
                                    % lab.numel(), lab).to(torch.int32)
                flic.flic_filter_relabel(h, stray, 10, num)
                torch.cuda.synchronize()
            flic.flic_filter_relabel(h, lab, 10, num)
            torch.cuda.synchronize()
            want, n = oracle.filter_relabel(
                oracle.label(f.range, s.elevation, s.az_step, 0.5, 3), 10)
            assert np.array_equal(lab.cpu().numpy(), want.reshape(-1)), k
            assert int(num.item()) == n, k
        assert flic.flic_device_status(h) == flic.FLIC_OK
    finally:
        h.close()
