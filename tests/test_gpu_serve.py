"""The server (continuous batching) on the GPU: every frame's result in a mixed stream of
range images and clouds from four sensors equals the same frame processed alone, and the
CPU oracle; a full admission queue refuses with FLIC_ERR_BUSY."""
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


def _alone(flic, f):
    """The frame through the single-frame calls."""
    s = f.sensor
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, f.delta, f.skip)
    try:
        lab = torch.empty(s.rows * s.cols, dtype=torch.int32, device="cuda")
        if f.xyz is None:
            flic.flic_label(h, torch.from_numpy(f.range.reshape(-1)).cuda(), lab)
            torch.cuda.synchronize()
            return lab.cpu().numpy()
        xyz = torch.from_numpy(f.xyz).cuda()
        rimg = torch.empty(s.rows * s.cols, dtype=torch.float32, device="cuda")
        pix = torch.empty(f.xyz.shape[0], dtype=torch.int32, device="cuda")
        plab = torch.empty_like(pix)
        flic.flic_project(h, xyz, rimg, pix)
        flic.flic_label(h, rimg, lab)
        flic.flic_scatter(h, lab, pix, plab)
        torch.cuda.synchronize()
        return plab.cpu().numpy()
    finally:
        h.close()


def _oracle(f):
    s = f.sensor
    if f.xyz is None:
        return oracle.label(f.range, s.elevation, s.az_step, f.delta, f.skip).reshape(-1)
    r, pix, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
    return oracle.scatter(oracle.label(r, s.elevation, s.az_step, f.delta, f.skip), pix)


def test_served_mix_equals_alone(flic):
    sensors = synth.c5_sensors()
    handles = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3) for s in sensors]
    frames = []
    for i in range(32):
        s = sensors[i % 4]
        frames.append((i % 4, synth.c5_frame(s, 5000 + i, as_cloud=(i // 4) % 2 == 1)))
    srv = flic.flic_server_create(handles, [260_001] * 4, nstreams=2, max_batch=16,
                                  mem_budget=256 << 20)
    try:
        outs = []
        flic.flic_server_hold(srv, True)  # the first 24 frames arrive together
        for i, (si, f) in enumerate(frames):
            if i == 24:
                flic.flic_server_hold(srv, False)  # the rest stream in behind them
            x = torch.from_numpy((f.range if f.xyz is None else f.xyz).reshape(-1)).pin_memory()
            n = f.range.size if f.xyz is None else f.xyz.shape[0]
            y = torch.full((n,), -77, dtype=torch.int32).pin_memory()
            assert flic.flic_server_submit(srv, si, 0 if f.xyz is None else 1, x, y, i) == flic.FLIC_OK
            outs.append((x, y))
        flic.flic_server_drain(srv, 60.0)
        recs = flic.flic_server_poll(srv)
        stats = flic.flic_server_stats(srv)
    finally:
        srv.close()
        for h in handles:
            h.close()
    assert sorted(r.tag for r in recs) == list(range(32))
    assert all(r.status == 0 for r in recs)
    assert stats["completed"] == 32 and stats["batches"] < 32  # frames were batched together
    assert max(r.batch_size for r in recs) > 1
    for (si, f), (_, y) in zip(frames, outs):
        got = y.numpy()
        np.testing.assert_array_equal(got, _alone(flic, f), err_msg=f.name)
        np.testing.assert_array_equal(got, _oracle(f), err_msg=f.name)


def test_full_queue_refuses(flic):
    s = synth.c5_sensors()[3]
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3)
    srv = flic.flic_server_create([h], [0], nstreams=1, max_batch=1, mem_budget=0, max_queue=2)
    try:
        f = synth.c5_frame(s, 42, as_cloud=False)
        x = torch.from_numpy(f.range.reshape(-1)).pin_memory()
        ys = [torch.empty(f.range.size, dtype=torch.int32).pin_memory() for _ in range(64)]
        sts = [flic.flic_server_submit(srv, 0, 0, x, ys[i], i) for i in range(64)]
        flic.flic_server_drain(srv, 60.0)
        recs = flic.flic_server_poll(srv)
        stats = flic.flic_server_stats(srv)
    finally:
        srv.close()
        h.close()
    assert flic.FLIC_ERR_BUSY in sts
    assert stats["rejected"] == sts.count(flic.FLIC_ERR_BUSY)
    assert len(recs) == sts.count(flic.FLIC_OK) == stats["completed"]
    want = oracle.label(f.range, s.elevation, s.az_step, 0.5, 3).reshape(-1)
    for r in recs:
        np.testing.assert_array_equal(ys[r.tag].numpy(), want)


def test_served_with_ground_extraction(flic):
    """Sensors whose handles have ground extraction on: the server's per-slot copies of the
    handles carry the setting, and every served frame (images and clouds) equals the
    oracle with the ground removed."""
    import math
    theta = math.radians(10.0)
    sensors = synth.c5_sensors()
    handles = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3) for s in sensors]
    for h in handles:
        flic.flic_set_ground(h, theta, 1.7)
    frames = [(i % 4, synth.c5_frame(sensors[i % 4], 7000 + i, as_cloud=(i // 4) % 2 == 1))
              for i in range(16)]
    srv = flic.flic_server_create(handles, [260_001] * 4, nstreams=2, max_batch=8,
                                  mem_budget=256 << 20)
    try:
        outs = []
        for i, (si, f) in enumerate(frames):
            x = torch.from_numpy((f.range if f.xyz is None else f.xyz).reshape(-1)).pin_memory()
            n = f.range.size if f.xyz is None else f.xyz.shape[0]
            y = torch.full((n,), -77, dtype=torch.int32).pin_memory()
            assert flic.flic_server_submit(srv, si, 0 if f.xyz is None else 1, x, y, i) == flic.FLIC_OK
            outs.append((x, y))  # the input stays alive until the frame completes
        flic.flic_server_drain(srv, 60.0)
        recs = flic.flic_server_poll(srv)
    finally:
        srv.close()
        for h in handles:
            h.close()
    assert sorted(r.tag for r in recs) == list(range(16)) and all(r.status == 0 for r in recs)
    for (si, f), (_, y) in zip(frames, outs):
        s = f.sensor
        if f.xyz is None:
            want = oracle.label_ground(f.range, s.elevation, s.az_step, 0.5, 3, True, theta, 1.7)
            want = want.reshape(-1)
        else:
            r, pix, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
            want = oracle.scatter(oracle.label_ground(r, s.elevation, s.az_step, 0.5, 3, True,
                                                      theta, 1.7), pix)
        np.testing.assert_array_equal(y.numpy(), want, err_msg=f.name)


def test_batch_of_more_clouds_than_one_projection_launch(flic):
    """104 clouds held and released as one batch: their projection and scatter run as two
    launches of items each (96 + 8); every cloud's point labels equal its alone result."""
    s = synth.c5_sensors()[0]
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3)
    clouds = [synth.c5_frame(s, 7000 + j, as_cloud=True) for j in range(4)]
    want = [_alone(flic, f) for f in clouds]
    mp = max(f.xyz.shape[0] for f in clouds)
    budget = 110 * (s.rows * s.cols * 8 + mp * 20)
    srv = flic.flic_server_create([h], [mp], nstreams=1, max_batch=128, mem_budget=budget)
    try:
        ins = [torch.from_numpy(f.xyz.reshape(-1)).pin_memory() for f in clouds]
        outs = []
        flic.flic_server_hold(srv, True)
        for i in range(104):
            y = torch.full((clouds[i % 4].xyz.shape[0],), -5, dtype=torch.int32).pin_memory()
            assert flic.flic_server_submit(srv, 0, 1, ins[i % 4], y, i) == flic.FLIC_OK
            outs.append(y)
        flic.flic_server_hold(srv, False)
        flic.flic_server_drain(srv, 60.0)
        recs = flic.flic_server_poll(srv)
    finally:
        srv.close()
        h.close()
    assert sorted(r.tag for r in recs) == list(range(104))
    assert all(r.status == 0 for r in recs)
    assert max(r.batch_size for r in recs) > 96
    for i, y in enumerate(outs):
        np.testing.assert_array_equal(y.numpy(), want[i % 4], err_msg=str(i))
