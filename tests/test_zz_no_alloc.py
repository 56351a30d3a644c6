"""flic_project_noalloc, the projection entry point for callers that cannot allocate
device memory (for example code inside a host framework whose GPU memory belongs to its
own pool).  It keeps its working memory in static arrays inside libflic, so these tests
check, through the C ABI, that its results equal flic_project's and the oracle's bit for
bit on two calls in a row (the second over a different, smaller frame, so leftovers of the
first call would show), that oversized frames are refused with a clear message, and that a
capturing stream is refused (its tables come from host arrays the next call overwrites).

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import ctypes

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


def _with_handle(flic, s, xyz):
    """The existing entry point: flic_project on a handle of the same geometry."""
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 1)
    try:
        rimg = torch.empty(s.rows * s.cols, dtype=torch.float32, device="cuda")
        pix = torch.empty(xyz.shape[0], dtype=torch.int32, device="cuda")
        flic.flic_project(h, xyz, rimg, pix)
        torch.cuda.synchronize()
        return rimg.cpu().numpy(), pix.cpu().numpy()
    finally:
        h.close()


def _no_alloc(flic, s, xyz):
    """The allocation-free entry point, called directly through the C ABI."""
    elev = np.ascontiguousarray(s.elevation, dtype=np.float64)
    rimg = torch.full((s.rows * s.cols,), -7.0, dtype=torch.float32, device="cuda")
    pix = torch.full((xyz.shape[0],), -9, dtype=torch.int32, device="cuda")
    st = flic._lib.flic_project_noalloc(
        s.rows, s.cols, elev.ctypes.data, float(s.az_step), xyz.data_ptr(), xyz.shape[0],
        rimg.data_ptr(), pix.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == flic.FLIC_OK, flic._lib.flic_last_error()
    torch.cuda.synchronize()
    return rimg.cpu().numpy(), pix.cpu().numpy()


def test_no_alloc_matches_flic_project_on_two_calls_in_a_row(flic):
    sensors = synth.c5_sensors()
    frames = [synth.c5_frame(sensors[3], 2001, as_cloud=True),   # 128 x 2048, the maximum
              synth.c5_frame(sensors[1], 2002, as_cloud=True)]   # 32 x 1024 after it
    for f in frames:
        xyz = torch.from_numpy(f.xyz).cuda()
        want_r, want_p = _with_handle(flic, f.sensor, xyz)
        got_r, got_p = _no_alloc(flic, f.sensor, xyz)
        np.testing.assert_array_equal(got_p, want_p)
        np.testing.assert_array_equal(got_r.view(np.uint32), want_r.view(np.uint32))
        assert (got_p >= 0).mean() > 0.9
        s = f.sensor
        r_o, pix_o, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
        np.testing.assert_array_equal(got_p, pix_o)
        np.testing.assert_array_equal(got_r.view(np.uint32), r_o.reshape(-1).view(np.uint32))


def test_no_alloc_refuses_frames_beyond_its_static_size(flic):
    rows, cols = 256, 2048  # 524,288 pixels > FLIC_NOALLOC_MAX_PIXELS
    elev = np.radians(np.linspace(20, -20, rows))
    out = torch.empty(rows * cols, dtype=torch.float32, device="cuda")
    st = flic._lib.flic_project_noalloc(rows, cols, elev.ctypes.data, 2 * np.pi / cols, None, 0,
                                       out.data_ptr(), None, None)
    assert st == flic.FLIC_ERR_INVALID
    assert b"static limits" in flic._lib.flic_last_error()


def test_no_alloc_refuses_a_capturing_stream(flic):
    s = synth.c5_sensors()[1]
    elev = np.ascontiguousarray(s.elevation, dtype=np.float64)
    out = torch.empty(s.rows * s.cols, dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        st = flic._lib.flic_project_noalloc(s.rows, s.cols, elev.ctypes.data, float(s.az_step),
                                           None, 0, out.data_ptr(), None, side.cuda_stream)
    assert st == flic.FLIC_ERR_UNSUPPORTED
    assert b"captured" in flic._lib.flic_last_error()
