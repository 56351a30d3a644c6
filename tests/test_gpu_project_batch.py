"""GPU parity of flic_project_batch / flic_scatter_batch: many clouds projected and scattered
by a few launches, each cloud equal to the oracle bit for bit (pixel map, range image,
labels, point labels) — c5 clouds with collisions on the four sensors, more clouds than one
launch takes, an empty cloud, the handles' own range buffers, agreement with the per-cloud
calls, and a repeated handle refused."""
import ctypes
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


def _handles(flic, frames):
    return [flic.flic_create(f.sensor.rows, f.sensor.cols, f.sensor.elevation, f.sensor.az_step,
                             f.delta, f.skip) for f in frames]


def _run(flic, frames, own_range=False):
    """Batched projection, batched labelling, batched scatter; results on the host."""
    hs = _handles(flic, frames)
    try:
        xyz = [torch.from_numpy(np.ascontiguousarray(f.xyz, np.float32).reshape(-1)).to(DEV)
               for f in frames]
        pix = [torch.full((f.xyz.shape[0],), -9, dtype=torch.int32, device=DEV) for f in frames]
        rimg = None if own_range else [torch.full((f.range.size,), -1.0, device=DEV)
                                       for f in frames]
        lab = [torch.full((f.range.size,), -5, dtype=torch.int32, device=DEV) for f in frames]
        plab = [torch.full_like(p, -7) for p in pix]
        args = flic.CloudArgs(hs, xyz, pix, range_out=rimg, labels=lab, point_labels=plab)
        flic.flic_project_batch(args)
        src = [flic.flic_range_buffer(h) for h in hs] if own_range else rimg
        b = flic.flic_batch_create(len(frames))
        try:
            flic.flic_label_batch(b, flic.BatchArgs(hs, src, lab))
            flic.flic_scatter_batch(args)
            torch.cuda.synchronize()
        finally:
            b.close()
        assert all(flic.flic_device_status(h) == flic.FLIC_OK for h in hs)
        return ([p.cpu().numpy() for p in pix],
                None if own_range else [r.cpu().numpy() for r in rimg],
                [x.cpu().numpy() for x in lab], [p.cpu().numpy() for p in plab])
    finally:
        for h in hs:
            h.close()


def _check(frames, pix, rimg, lab, plab):
    for i, f in enumerate(frames):
        s = f.sensor
        r_o, pix_o, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
        msg = f"cloud {i} ({f.name})"
        np.testing.assert_array_equal(pix[i], pix_o, err_msg=msg)
        if rimg is not None:
            np.testing.assert_array_equal(rimg[i].view(np.uint32),
                                          r_o.reshape(-1).view(np.uint32), err_msg=msg)
        lab_o = oracle.label(r_o, s.elevation, s.az_step, f.delta, f.skip)
        np.testing.assert_array_equal(lab[i], lab_o.reshape(-1), err_msg=msg)
        np.testing.assert_array_equal(plab[i], oracle.scatter(lab_o, pix_o), err_msg=msg)


def test_c5_clouds_on_four_sensors(flic):
    sens = synth.c5_sensors()
    frames = [synth.c5_frame(sens[i % 4], 8100 + i, as_cloud=True) for i in range(12)]
    _check(frames, *_run(flic, frames))


def test_handles_own_range_buffers(flic):
    sens = synth.c5_sensors()
    frames = [synth.c5_frame(sens[(i + 1) % 4], 8150 + i, as_cloud=True) for i in range(6)]
    _check(frames, *_run(flic, frames, own_range=True))


def test_more_clouds_than_one_launch_and_an_empty_cloud(flic):
    sens = synth.c5_sensors()
    base = [synth.c5_frame(sens[j % 2], 8200 + j, as_cloud=True) for j in range(5)]
    frames = [base[i % 5] for i in range(100)]
    s = sens[1]
    empty = synth.Frame(s, np.zeros((s.rows, s.cols), np.float32), 0.5, 3, None,
                        xyz=np.zeros((0, 3), np.float32), name="empty")
    frames[37] = empty
    pix, rimg, lab, plab = _run(flic, frames)
    assert pix[37].shape == (0,) and plab[37].shape == (0,)
    assert not np.any(rimg[37]) and np.all(lab[37] == -1)
    keep = [i for i in range(100) if i != 37]
    # identical clouds give identical results wherever they sit in the launches
    for i in keep:
        j = i % 5
        for v in (pix, rimg, lab, plab):
            np.testing.assert_array_equal(v[i], v[j], err_msg=f"cloud {i}")
    _check(base, *[[v[j] for j in range(5)] for v in (pix, rimg, lab, plab)])
    _check([frames[96], frames[99]], *[[v[96], v[99]] for v in (pix, rimg, lab, plab)])


def test_equals_the_per_cloud_calls(flic):
    sens = synth.c5_sensors()
    frames = [synth.c5_frame(sens[i], 8250 + i, as_cloud=True) for i in range(4)]
    pix_b, rimg_b, lab_b, plab_b = _run(flic, frames)
    for i, f in enumerate(frames):
        s = f.sensor
        h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, f.delta, f.skip)
        try:
            x = torch.from_numpy(np.ascontiguousarray(f.xyz, np.float32).reshape(-1)).to(DEV)
            r = torch.empty(s.rows * s.cols, device=DEV)
            p = torch.empty(f.xyz.shape[0], dtype=torch.int32, device=DEV)
            flic.flic_project(h, x, r, p)
            lab = torch.empty(s.rows * s.cols, dtype=torch.int32, device=DEV)
            flic.flic_label(h, r, lab)
            q = torch.empty_like(p)
            flic.flic_scatter(h, lab, p, q)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(p.cpu().numpy(), pix_b[i])
            np.testing.assert_array_equal(r.cpu().numpy().view(np.uint32), rimg_b[i].view(np.uint32))
            np.testing.assert_array_equal(q.cpu().numpy(), plab_b[i])
        finally:
            h.close()


def test_repeated_handle_and_null_arguments_are_refused(flic):
    s = synth.c5_sensors()[1]
    f = synth.c5_frame(s, 8300, as_cloud=True)
    h = flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3)
    try:
        x = torch.from_numpy(f.xyz.reshape(-1)).to(DEV)
        p = torch.empty(f.xyz.shape[0], dtype=torch.int32, device=DEV)
        with pytest.raises(ValueError):
            flic.CloudArgs([h, h], [x, x], [p, p])
        hs = (ctypes.c_void_p * 2)(h.ptr, h.ptr)
        xs = (ctypes.c_void_p * 2)(x.data_ptr(), x.data_ptr())
        ps = (ctypes.c_void_p * 2)(p.data_ptr(), p.data_ptr())
        ns = (ctypes.c_int64 * 2)(f.xyz.shape[0], f.xyz.shape[0])
        st = flic._lib.flic_project_batch(hs, 2, xs, ns, None, ps, None)
        assert st == flic.FLIC_ERR_INVALID
        st = flic._lib.flic_scatter_batch(hs, 2, xs, ps, ns, ps, None)
        assert st == flic.FLIC_ERR_INVALID
        one = (ctypes.c_void_p * 1)(h.ptr)
        assert flic._lib.flic_project_batch(one, 1, None, ns, None, ps, None) == flic.FLIC_ERR_INVALID
        assert flic._lib.flic_project_batch(one, -1, xs, ns, None, ps, None) == flic.FLIC_ERR_INVALID
        assert flic._lib.flic_project_batch(None, 0, None, None, None, None, None) == flic.FLIC_OK
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
    finally:
        h.close()


def _cloud_at(g, elev, C, n, on_bounds, near=False):
    """Points in all directions of the sensor's field; on_bounds puts half of them on the
    exact column boundary angles c * 2pi / C and on the midpoints between beams; near puts
    them at log-spaced angular distances 1e-8 .. 1e-3 rad either side of a column boundary
    and of a row boundary (the outer ones included)."""
    es = np.sort(elev)
    lo = es[0] - (es[1] - es[0]) / 2 - 0.02
    hi = es[-1] + (es[-1] - es[-2]) / 2 + 0.02
    el = g.uniform(lo, hi, n)
    az = g.uniform(0, 2 * math.pi, n)
    if on_bounds:
        k = n // 2
        az[:k] = g.integers(0, C, k) * (2 * math.pi / C)
        j = g.integers(1, len(es), k)
        el[:k // 2] = (es[j[:k // 2] - 1] + es[j[:k // 2]]) / 2
    if near:
        bounds = np.concatenate([[es[0] - (es[1] - es[0]) / 2], (es[1:] + es[:-1]) / 2,
                                 [es[-1] + (es[-1] - es[-2]) / 2]])
        dist = 10.0 ** g.uniform(-8, -3, n) * g.choice([-1.0, 1.0], n)
        az = g.integers(0, C, n) * (2 * math.pi / C) + dist
        el = bounds[g.integers(0, len(bounds), n)] + \
            10.0 ** g.uniform(-8, -3, n) * g.choice([-1.0, 1.0], n)
        az[: n // 3] = g.uniform(0, 2 * math.pi, n // 3)        # row boundaries alone
        el[n // 3: 2 * n // 3] = g.uniform(lo, hi, n - n // 3 - n // 3)[: n // 3]
    d = g.uniform(0.5, 120, n)
    xyz = np.stack([d * np.cos(el) * np.cos(az), d * np.cos(el) * np.sin(az), d * np.sin(el)], 1)
    xyz = xyz.astype(np.float32)
    xyz[::53] = 0.0
    return xyz


@pytest.mark.parametrize("case", ["wide_field_bisection", "16384_cols", "unsorted_rows",
                                  "two_rows", "boundaries", "near_boundaries",
                                  "near_boundaries_16384", "near_boundaries_16"])
def test_row_and_column_seeds(flic, case):
    """The row search seeded from tan(elevation) buckets (bisection where a boundary lies
    beyond 80 degrees), the column search from the polynomial azimuth: same pixels and
    ranges as the oracle's linear row scan and double-precision azimuth seed."""
    g = np.random.default_rng(sum(map(ord, case)))
    R, C = {"wide_field_bisection": (32, 1024), "16384_cols": (128, 16384),
            "unsorted_rows": (64, 2048), "two_rows": (2, 1800), "boundaries": (64, 2048),
            "near_boundaries": (128, 2048), "near_boundaries_16384": (64, 16384),
            "near_boundaries_16": (16, 1800)}[case]
    if case == "wide_field_bisection":
        elev = np.radians(np.linspace(-84.0, 84.0, R))
    elif case == "two_rows":
        elev = np.radians(np.array([-1.0, 2.0]))
    else:
        elev = np.radians(np.linspace(-24.9, 15.1, R) + g.uniform(-0.05, 0.05, R))
    if case == "unsorted_rows":
        elev = g.permutation(elev)
    xyz = _cloud_at(g, elev, C, 400_000, case == "boundaries", case.startswith("near"))
    h = flic.flic_create(R, C, elev, 2 * math.pi / C, 0.5, 2)
    try:
        x = torch.from_numpy(xyz.reshape(-1)).to(DEV)
        r = torch.empty(R * C, device=DEV)
        p = torch.empty(xyz.shape[0], dtype=torch.int32, device=DEV)
        flic.flic_project(h, x, r, p)
        torch.cuda.synchronize()
        assert flic.flic_device_status(h) == flic.FLIC_OK
        r_o, pix_o, _ = oracle.project(xyz, R, C, elev, 2 * math.pi / C)
        np.testing.assert_array_equal(p.cpu().numpy(), pix_o)
        np.testing.assert_array_equal(r.cpu().numpy().view(np.uint32),
                                      r_o.reshape(-1).view(np.uint32))
        assert (pix_o >= 0).mean() > (0.3 if case.startswith("near") else 0.5)
    finally:
        h.close()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 1001, 40_003])
def test_unaligned_and_ragged_clouds(flic, n):
    """Clouds whose xyz, point_pixel or range_out start off their 16-byte (8-byte)
    boundary take the one-point / one-pixel paths; counts that are not a multiple of four
    leave a tail: every combination equal to the oracle, single and batched."""
    s = synth.c5_sensors()[2]
    f = synth.c5_frame(s, 8400 + n, as_cloud=True)
    xyz = np.ascontiguousarray(f.xyz[:n])
    r_o, pix_o, _ = oracle.project(xyz, s.rows, s.cols, s.elevation, s.az_step)
    hs = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3) for _ in range(4)]
    try:
        bufs = []
        for off in range(4):  # offset in elements from a 256-byte aligned allocation
            xb = torch.zeros(3 * n + 3 * off + 4, device=DEV)
            xb[3 * off:3 * off + 3 * n] = torch.from_numpy(xyz.reshape(-1)).to(DEV)
            pb = torch.full((n + off + 4,), -9, dtype=torch.int32, device=DEV)
            rb = torch.full((s.rows * s.cols + off,), -1.0, device=DEV)
            bufs.append((xb, pb, rb, off))
        # single-cloud calls: xyz offset 3*off floats, point_pixel and range_out off floats
        for (xb, pb, rb, off), h in zip(bufs, hs):
            st = flic._lib.flic_project(h.ptr, xb.data_ptr() + 12 * off, n,
                                        rb.data_ptr() + 4 * off, pb.data_ptr() + 4 * off, None)
            assert st == flic.FLIC_OK
        torch.cuda.synchronize()
        for (xb, pb, rb, off), h in zip(bufs, hs):
            assert flic.flic_device_status(h) == flic.FLIC_OK
            np.testing.assert_array_equal(pb.cpu().numpy()[off:off + n], pix_o, err_msg=f"off {off}")
            assert np.all(pb.cpu().numpy()[off + n:] == -9) and np.all(pb.cpu().numpy()[:off] == -9)
            np.testing.assert_array_equal(rb.cpu().numpy()[off:].view(np.uint32),
                                          r_o.reshape(-1).view(np.uint32), err_msg=f"off {off}")
        # the same four clouds as one batch
        for xb, pb, rb, off in bufs:
            pb.fill_(-9)
            rb.fill_(-1.0)
        k = 4
        h_arr = (ctypes.c_void_p * k)(*[h.ptr for h in hs])
        x_arr = (ctypes.c_void_p * k)(*[xb.data_ptr() + 12 * off for xb, _, _, off in bufs])
        p_arr = (ctypes.c_void_p * k)(*[pb.data_ptr() + 4 * off for _, pb, _, off in bufs])
        r_arr = (ctypes.c_void_p * k)(*[rb.data_ptr() + 4 * off for _, _, rb, off in bufs])
        n_arr = (ctypes.c_int64 * k)(*([n] * k))
        assert flic._lib.flic_project_batch(h_arr, k, x_arr, n_arr, r_arr, p_arr, None) == flic.FLIC_OK
        torch.cuda.synchronize()
        for xb, pb, rb, off in bufs:
            np.testing.assert_array_equal(pb.cpu().numpy()[off:off + n], pix_o, err_msg=f"off {off}")
            np.testing.assert_array_equal(rb.cpu().numpy()[off:].view(np.uint32),
                                          r_o.reshape(-1).view(np.uint32), err_msg=f"off {off}")
    finally:
        for h in hs:
            h.close()


def test_consecutive_projections_on_the_same_handles(flic):
    """Every decode leaves a handle's keys empty: batched and single projections of
    different clouds on the same handles, one after another with no clearing between
    them, each equal to the oracle."""
    sens = synth.c5_sensors()
    hs = [flic.flic_create(s.rows, s.cols, s.elevation, s.az_step, 0.5, 3) for s in sens]
    try:
        for rnd in range(4):
            frames = [synth.c5_frame(sens[i], 8500 + 10 * rnd + i, as_cloud=True) for i in range(4)]
            xyz = [torch.from_numpy(f.xyz.reshape(-1)).to(DEV) for f in frames]
            pix = [torch.empty(f.xyz.shape[0], dtype=torch.int32, device=DEV) for f in frames]
            rng = [torch.empty(f.range.size, device=DEV) for f in frames]
            if rnd % 2 == 0:
                flic.flic_project_batch(flic.CloudArgs(hs, xyz, pix, range_out=rng))
            else:
                for h, x, r, p in zip(hs, xyz, rng, pix):
                    flic.flic_project(h, x, r, p)
            torch.cuda.synchronize()
            for f, p, r in zip(frames, pix, rng):
                s = f.sensor
                r_o, pix_o, _ = oracle.project(f.xyz, s.rows, s.cols, s.elevation, s.az_step)
                np.testing.assert_array_equal(p.cpu().numpy(), pix_o, err_msg=f"round {rnd}")
                np.testing.assert_array_equal(r.cpu().numpy().view(np.uint32),
                                              r_o.reshape(-1).view(np.uint32), err_msg=f"round {rnd}")
        assert all(flic.flic_device_status(h) == flic.FLIC_OK for h in hs)
    finally:
        for h in hs:
            h.close()
