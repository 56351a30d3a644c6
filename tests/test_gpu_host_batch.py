"""flic_label_batch_host: frames labelled from packed host buffers, with the copies of one
group of frames overlapping the labelling of another.  Every frame's labels equal the
oracle's (and the device-buffer batch path's), for any number of groups."""
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


def _handles(flic, frames):
    return [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                             f.delta, f.skip) for f in frames]


def _want(frames, idx):
    return {i: oracle.label(frames[i].range, frames[i].sensor.elevation, frames[i].sensor.az_step,
                            frames[i].delta, frames[i].skip).reshape(-1) for i in idx}


def _packed(frames, pin=True):
    host = torch.from_numpy(np.concatenate([f.range.reshape(-1) for f in frames]))
    out = torch.full((host.numel(),), -7, dtype=torch.int32)
    return (host.pin_memory(), out.pin_memory()) if pin else (host, out)


def _split(out, frames):
    offs = np.cumsum([0] + [f.range.size for f in frames])
    o = out.numpy()
    return [o[offs[i]:offs[i + 1]] for i in range(len(frames))]


@pytest.mark.parametrize("ready", [False, True])
@pytest.mark.parametrize("groups", [0, 1, 2, 3, 7, 16])
def test_c4_groups(flic, groups, ready):
    frames = synth.config_c4(48)
    hs = _handles(flic, frames)
    try:
        host, out = _packed(frames)
        b = flic.flic_batch_create(len(frames))
        flic.flic_label_batch_host(b, hs, host, out, groups, ready)
        torch.cuda.synchronize()
        got = _split(out, frames)
        want = _want(frames, range(len(frames)))
        for i in range(len(frames)):
            assert np.array_equal(got[i], want[i]), (groups, i)
        b.close()
        for h in hs:
            assert flic.flic_device_status(h) == flic.FLIC_OK
    finally:
        for h in hs:
            h.close()


def test_matches_device_batch_and_repeats(flic):
    """The full 256-frame batch: equal to flic_label_batch on device buffers; repeated
    calls (graph replay in every group) and a call with new inputs stay exact."""
    frames = synth.config_c4(256)
    hs = _handles(flic, frames)
    try:
        host, out = _packed(frames)
        rs = [torch.from_numpy(f.range.reshape(-1)).to(DEV) for f in frames]
        ls = [torch.empty(f.range.size, dtype=torch.int32, device=DEV) for f in frames]
        bd = flic.flic_batch_create(len(frames))
        flic.flic_label_batch(bd, flic.BatchArgs(hs, rs, ls))
        b = flic.flic_batch_create(len(frames))
        for rep in range(3):
            out.fill_(-7)
            flic.flic_label_batch_host(b, hs, host, out, input_ready=rep == 2)
            torch.cuda.synchronize()
            got = _split(out, frames)
            for i in range(len(frames)):
                assert np.array_equal(got[i], ls[i].cpu().numpy()), (rep, i)
        want = _want(frames, (0, 1, 100, 255))
        for i, w in want.items():
            assert np.array_equal(got[i], w), i
        # new readings in the same buffers: every frame mirrored left-right
        for f in frames:
            f.range[:] = np.ascontiguousarray(f.range[:, ::-1])
        host.copy_(torch.from_numpy(np.concatenate([f.range.reshape(-1) for f in frames])))
        flic.flic_label_batch_host(b, hs, host, out, 5)
        torch.cuda.synchronize()
        got = _split(out, frames)
        for i, w in _want(frames, (3, 64, 200)).items():
            assert np.array_equal(got[i], w), i
        b.close()
        bd.close()
    finally:
        for h in hs:
            h.close()


def test_pageable_and_numpy_buffers(flic):
    frames = synth.config_c4(12)
    hs = _handles(flic, frames)
    try:
        host, out = _packed(frames, pin=False)
        b = flic.flic_batch_create(16)
        flic.flic_label_batch_host(b, hs, host, out, 3)
        torch.cuda.synchronize()
        want = _want(frames, range(len(frames)))
        for i, g in enumerate(_split(out, frames)):
            assert np.array_equal(g, want[i]), i
        hn = host.numpy().copy()
        on = np.full(hn.size, -7, np.int32)
        flic.flic_label_batch_host(b, hs, hn, on, 2)
        torch.cuda.synchronize()
        assert np.array_equal(on, out.numpy())
        b.close()
    finally:
        for h in hs:
            h.close()


def test_growth_shared_handle_and_tuning(flic):
    """A larger batch after a smaller one (device copies grown), one handle for every
    frame, a tuning change in between: still exact."""
    f = synth.config_c1()
    R, C = f.sensor.rows, f.sensor.cols
    h = flic.flic_create(R, C, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
    try:
        b = flic.flic_batch_create(9)
        for n, tuning in ((2, None), (9, (4096, 256, 0, 0)), (5, (0, 0, 0, 0))):
            if tuning:
                flic.flic_batch_set_tuning(b, *tuning)
            ranges = [np.ascontiguousarray(np.roll(f.range, 13 * i, axis=1)) for i in range(n)]
            host = torch.from_numpy(np.concatenate([x.reshape(-1) for x in ranges])).pin_memory()
            out = torch.empty(host.numel(), dtype=torch.int32).pin_memory()
            flic.flic_label_batch_host(b, [h] * n, host, out, 4)
            torch.cuda.synchronize()
            o = out.numpy()
            for i, x in enumerate(ranges):
                want = oracle.label(x, f.sensor.elevation, f.sensor.az_step, f.delta, f.skip)
                assert np.array_equal(o[i * R * C:(i + 1) * R * C], want.reshape(-1)), (n, i)
        b.close()
    finally:
        h.close()


def test_errors(flic):
    f = synth.config_c1()
    h = flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                         f.delta, f.skip)
    try:
        b = flic.flic_batch_create(2)
        n = f.range.size
        host = torch.from_numpy(f.range.reshape(-1).copy())
        out = torch.empty(n, dtype=torch.int32)
        with pytest.raises(flic.FlicError) as e:
            flic.flic_label_batch_host(b, [h, h, h], torch.zeros(3 * n), torch.empty(3 * n, dtype=torch.int32))
        assert e.value.status == flic.FLIC_ERR_BUSY
        with pytest.raises(flic.FlicError) as e:
            flic.flic_label_batch_host(b, [h], host, out, 17)
        assert e.value.status == flic.FLIC_ERR_INVALID
        hs1 = (flic.ctypes.c_void_p * 1)(h.ptr)
        st = flic._lib.flic_label_batch_host(b.ptr, hs1, 1, host.data_ptr(), out.data_ptr(), 0,
                                             4, None)
        assert st == flic.FLIC_ERR_INVALID  # unknown flag
        # overlapping buffers: the labels would overwrite readings not yet uploaded
        both = torch.zeros(2 * n, dtype=torch.int32)
        with pytest.raises(flic.FlicError) as e:
            flic.flic_label_batch_host(b, [h], both[:n].view(torch.float32), both[n // 2:n // 2 + n])
        assert e.value.status == flic.FLIC_ERR_INVALID
        with pytest.raises(ValueError):
            flic.flic_label_batch_host(b, [h], host.to(DEV), out)
        flic.flic_label_batch_host(b, [], host[:0], out[:0])  # nothing to do
        b.close()
    finally:
        h.close()


def test_input_ready_back_to_back(flic):
    """Calls queued back to back with FLIC_HOST_INPUT_READY, each on its own input and
    output buffers, alternate between the object's two sides and overlap on the GPU: every
    output holds its own input's labels."""
    frames = synth.config_c4(64)
    hs = _handles(flic, frames)
    try:
        base = [f.range.copy() for f in frames]
        ins, outs, wants = [], [], []
        for v in range(5):
            ranges = [np.ascontiguousarray(np.roll(x, 17 * v, axis=1)) for x in base]
            ins.append(torch.from_numpy(np.concatenate([x.reshape(-1) for x in ranges])).pin_memory())
            outs.append(torch.full((ins[-1].numel(),), -7, dtype=torch.int32).pin_memory())
            wants.append(ranges)
        b = flic.flic_batch_create(len(frames))
        stream = torch.cuda.Stream()
        for rep in range(2):
            for v in range(5):
                flic.flic_label_batch_host(b, hs, ins[v], outs[v], 3, True, stream)
            stream.synchronize()
            for v in range(5):
                got = _split(outs[v], frames)
                for i in (0, 9, 31, 63):
                    f = frames[i]
                    want = oracle.label(wants[v][i], f.sensor.elevation, f.sensor.az_step,
                                        f.delta, f.skip)
                    assert np.array_equal(got[i], want.reshape(-1)), (rep, v, i)
        b.close()
    finally:
        for h in hs:
            h.close()


def test_ordered_after_stream_work(flic):
    """Without the flag the call follows the work queued on the stream: readings written
    into the pinned input by a device-to-host copy queued just before are the ones
    labelled."""
    frames = synth.config_c4(16)
    hs = _handles(flic, frames)
    try:
        host, out = _packed(frames)
        dev = host.to(DEV)
        host.zero_()  # the labels of zeros would be all -1
        b = flic.flic_batch_create(len(frames))
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        torch.cuda._sleep(20_000_000)  # keep the stream busy for a while
        host.copy_(dev, non_blocking=True)
        flic.flic_label_batch_host(b, hs, host, out, 2, False, stream)
        torch.cuda.synchronize()
        want = _want(frames, range(len(frames)))
        for i, g in enumerate(_split(out, frames)):
            assert np.array_equal(g, want[i]), i
        b.close()
    finally:
        for h in hs:
            h.close()
