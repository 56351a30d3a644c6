"""Thin Python binding of libflic (include/flic.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device buffers are torch
tensors on the CUDA device (PyTorch provides memory and streams only); every step of the
hot path runs in libflic's kernels.  Importing this module loads libflic.so and raises
if it has not been built (``python -c "import __graft_entry__ as g; g.build()"``):
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import typing

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libflic.so")

FLIC_OK = 0
FLIC_ERR_INVALID = 1
FLIC_ERR_OOM = 2
FLIC_ERR_CUDA = 3
FLIC_ERR_TIMEOUT = 4
FLIC_ERR_BUSY = 5
FLIC_ERR_UNSUPPORTED = 6
FLIC_FLAG_NO_WRAP = 1
FLIC_FLAG_EXACT_RAY = 2
FLIC_FLAG_SUBLATTICE = 4
FLIC_FLAG_DIAGONAL = 8
FLIC_HOST_INPUT_READY = 1
FLIC_MAX_PIXELS = 1 << 21
FLIC_MAX_ROWS = 512
FLIC_MAX_SKIP = 8
FLIC_NOALLOC_MAX_PIXELS = 1 << 18
FLIC_NOALLOC_MAX_COLS = 8192

# every symbol include/flic.h declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_F32 = ctypes.c_float
_F64 = ctypes.c_double
SIGNATURES = {
    "flic_abi_version": (_I32, []),
    "flic_last_error": (ctypes.c_char_p, []),
    "flic_create": (_I32, [_I32, _I32, _P, _F64, _F32, _I32, _P]),
    "flic_create_ex": (_I32, [_I32, _I32, _P, _F64, _F32, _I32, _U32, _P]),
    "flic_destroy": (_I32, [_P]),
    "flic_get_tables": (_I32, [_P, _P, _P]),
    "flic_get_diag_table": (_I32, [_P, _P]),
    "flic_project_batch": (_I32, [_P, _I32, _P, _P, _P, _P, _P]),
    "flic_scatter_batch": (_I32, [_P, _I32, _P, _P, _P, _P, _P]),
    "flic_edges": (_I32, [_P, _P, _P, _P]),
    "flic_label": (_I32, [_P, _P, _P, _P]),
    "flic_project": (_I32, [_P, _P, _I64, _P, _P, _P]),
    "flic_range_buffer": (_P, [_P]),
    "flic_scatter": (_I32, [_P, _P, _P, _I64, _P, _P]),
    "flic_set_ground": (_I32, [_P, _F64, _F64]),
    "flic_filter_relabel": (_I32, [_P, _P, _I32, _P, _P]),
    "flic_filter_relabel_batch": (_I32, [_P, _P, _P, _I32, _I32, _P, _P]),
    "flic_label_filter_batch": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _P]),
    "flic_batch_create": (_I32, [_I32, _P]),
    "flic_label_batch": (_I32, [_P, _P, _P, _P, _I32, _P]),
    "flic_label_batch_host": (_I32, [_P, _P, _I32, _P, _P, _I32, _U32, _P]),
    "flic_batch_destroy": (_I32, [_P]),
    "flic_set_tuning": (_I32, [_P, _I32, _I32, _I32]),
    "flic_batch_set_tuning": (_I32, [_P, _I32, _I32, _I32, _I32]),
    "flic_batch_set_schedule": (_I32, [_P, _I32]),
    "flic_plan_info": (_I32, [_P, _P]),
    "flic_plan_frame": (_I32, [_I32, _I32, _I32, _I32, _I32, _P]),
    "flic_batch_last_plan": (_I32, [_P, _P]),
    "flic_device_status": (_I32, [_P, _I32]),
    "flic_debug_set_iter_limit": (_I32, [_P, _I32]),
    "flic_project_noalloc": (_I32, [_I32, _I32, _P, _F64, _P, _I64, _P, _P, _P]),
    "flic_server_create": (_I32, [_P, _I32, _P, _I32, _I32, _I64, _I32, _P]),
    "flic_server_submit": (_I32, [_P, _I32, _I32, _P, _I64, _P, ctypes.c_uint64]),
    "flic_server_poll": (_I32, [_P, _P, _I32]),
    "flic_server_hold": (_I32, [_P, _I32]),
    "flic_server_drain": (_I32, [_P, _F64]),
    "flic_server_stats": (_I32, [_P, _P]),
    "flic_server_destroy": (_I32, [_P]),
    "flic_server_clock": (_F64, []),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libflic.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class FlicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libflic status {status}: {message}")
        self.status = status


def _check(st: int) -> None:
    if st != FLIC_OK:
        raise FlicError(st, (_lib.flic_last_error() or b"").decode())


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype_name: str, numel: int | None = None, what: str = "tensor") -> int:
    """Device pointer of a contiguous CUDA tensor of the given dtype (and size)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"{what} must be {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Handle:
    """A flic_handle plus the shape it was created with (closing is explicit or at GC)."""

    def __init__(self, ptr: int, rows: int, cols: int, skip: int, delta: float, wrap: bool):
        self.ptr = ptr
        self.rows, self.cols, self.skip, self.delta, self.wrap = rows, cols, skip, delta, wrap

    @property
    def npix(self) -> int:
        return self.rows * self.cols

    def close(self) -> None:
        if self.ptr:
            ptr, self.ptr = self.ptr, None  # freed even when the call reports an error
            _check(_lib.flic_destroy(ptr))

    def __del__(self):
        try:
            if self.ptr:
                _lib.flic_destroy(self.ptr)
        except Exception:
            pass


def flic_abi_version() -> int:
    return _lib.flic_abi_version()


def flic_create(rows: int, cols: int, elevation, az_step: float, delta: float, skip: int,
                wrap: bool = True, exact_ray: bool = False, lattice: bool = False,
                diagonal: bool = False) -> Handle:
    """lattice: the paper's sparse Map Connection (every skip-th point joined at offset
    skip, direct neighbours everywhere) instead of offsets 1..skip from every pixel;
    diagonal: the diagonal Map Connections (r, c)-(r+k, c+-k), k = 1..skip, as well."""
    elev = np.ascontiguousarray(elevation, dtype=np.float64)
    if elev.shape != (rows,):
        raise ValueError("elevation must have one entry per row")
    out = ctypes.c_void_p()
    flags = ((0 if wrap else FLIC_FLAG_NO_WRAP) | (FLIC_FLAG_EXACT_RAY if exact_ray else 0)
             | (FLIC_FLAG_SUBLATTICE if lattice else 0) | (FLIC_FLAG_DIAGONAL if diagonal else 0))
    _check(_lib.flic_create_ex(rows, cols, elev.ctypes.data, float(az_step), float(delta), skip,
                               flags, ctypes.byref(out)))
    return Handle(out.value, rows, cols, skip, float(np.float32(delta)), wrap)


def flic_destroy(h: Handle) -> None:
    h.close()


def flic_get_tables(h: Handle):
    kv = np.zeros((h.rows, h.skip), np.float32)
    kh = np.zeros((h.rows, h.skip), np.float32)
    _check(_lib.flic_get_tables(h.ptr, kv.ctypes.data, kh.ctypes.data))
    return kv, kh


def flic_get_diag_table(h: Handle):
    kd = np.zeros((h.rows, h.skip), np.float32)
    _check(_lib.flic_get_diag_table(h.ptr, kd.ctypes.data))
    return kd


def flic_plan_info(h: Handle) -> dict:
    info = np.zeros(5, np.int32)
    _check(_lib.flic_plan_info(h.ptr, info.ctypes.data))
    return dict(strips=int(info[0]), strip_w=int(info[1]), pitch=int(info[2]),
                smem=int(info[3]), threads=int(info[4]))


def flic_plan_frame(rows: int, cols: int, skip: int, px_per_cta: int = 16384,
                    max_strips: int = 64) -> dict:
    """Host-only strip split (no GPU needed)."""
    info = np.zeros(4, np.int32)
    _check(_lib.flic_plan_frame(rows, cols, skip, px_per_cta, max_strips, info.ctypes.data))
    return dict(strips=int(info[0]), strip_w=int(info[1]), pitch=int(info[2]), smem=int(info[3]))


def flic_set_tuning(h: Handle, px_per_cta: int = 0, threads: int = 0, max_strips: int = 0) -> None:
    _check(_lib.flic_set_tuning(h.ptr, px_per_cta, threads, max_strips))


def flic_edges(h: Handle, range_img, mask, stream=None) -> None:
    _check(_lib.flic_edges(h.ptr, _dptr(range_img, "float32", h.npix, "range"),
                           _dptr(mask, "int16", h.npix, "mask"), _stream(stream)))


def flic_label(h: Handle, range_img, labels, stream=None) -> None:
    _check(_lib.flic_label(h.ptr, _dptr(range_img, "float32", h.npix, "range"),
                           _dptr(labels, "int32", h.npix, "labels"), _stream(stream)))


def flic_project(h: Handle, xyz, range_out, point_pixel, stream=None) -> None:
    n = 0 if isinstance(xyz, int) else xyz.numel() // 3
    if not isinstance(xyz, int) and xyz.numel() != 3 * n:
        raise ValueError("xyz must hold n*3 floats")
    _check(_lib.flic_project(h.ptr, _dptr(xyz, "float32", None, "xyz"), n,
                             _dptr(range_out, "float32", h.npix, "range_out"),
                             _dptr(point_pixel, "int32", n, "point_pixel"), _stream(stream)))


class CloudArgs:
    """Host pointer arrays for flic_project_batch / flic_scatter_batch (one distinct handle
    per cloud), built once and reusable across calls."""

    def __init__(self, handles, xyz, point_pixel, range_out=None, labels=None,
                 point_labels=None):
        k = len(handles)
        if len({h.ptr for h in handles}) != k:
            raise ValueError("every cloud needs its own handle")
        self.n = k
        self.hs = (ctypes.c_void_p * k)(*[h.ptr for h in handles])
        counts = [x.numel() // 3 for x in xyz]
        self.counts = (ctypes.c_int64 * k)(*counts)
        self.xyz = (ctypes.c_void_p * k)(*[_dptr(x, "float32", 3 * c, "xyz")
                                           for x, c in zip(xyz, counts)])
        self.pix = (ctypes.c_void_p * k)(*[_dptr(p, "int32", c, "point_pixel")
                                           for p, c in zip(point_pixel, counts)])
        self.rng = None if range_out is None else (ctypes.c_void_p * k)(
            *[_dptr(r, "float32", h.npix, "range_out") for r, h in zip(range_out, handles)])
        self.lab = None if labels is None else (ctypes.c_void_p * k)(
            *[_dptr(l, "int32", h.npix, "labels") for l, h in zip(labels, handles)])
        self.plab = None if point_labels is None else (ctypes.c_void_p * k)(
            *[_dptr(p, "int32", c, "point_labels") for p, c in zip(point_labels, counts)])
        self._keep = (handles, xyz, point_pixel, range_out, labels, point_labels)


def flic_project_batch(args: CloudArgs, stream=None) -> None:
    _check(_lib.flic_project_batch(args.hs, args.n, args.xyz, args.counts, args.rng, args.pix,
                                   _stream(stream)))


def flic_scatter_batch(args: CloudArgs, stream=None) -> None:
    if args.lab is None or args.plab is None:
        raise ValueError("flic_scatter_batch needs labels and point_labels")
    _check(_lib.flic_scatter_batch(args.hs, args.n, args.lab, args.pix, args.counts, args.plab,
                                   _stream(stream)))


def flic_range_buffer(h: Handle) -> int:
    return _lib.flic_range_buffer(h.ptr)


def flic_scatter(h: Handle, labels, point_pixel, point_labels, stream=None) -> None:
    n = point_pixel.numel()
    _check(_lib.flic_scatter(h.ptr, _dptr(labels, "int32", h.npix, "labels"),
                             _dptr(point_pixel, "int32", n, "point_pixel"), n,
                             _dptr(point_labels, "int32", n, "point_labels"), _stream(stream)))


class Batch:
    def __init__(self, ptr: int, max_frames: int):
        self.ptr = ptr
        self.max_frames = max_frames

    def close(self) -> None:
        if self.ptr:
            ptr, self.ptr = self.ptr, None  # freed even when the call reports an error
            _check(_lib.flic_batch_destroy(ptr))

    def __del__(self):
        try:
            if self.ptr:
                _lib.flic_batch_destroy(self.ptr)
        except Exception:
            pass


def flic_batch_create(max_frames: int) -> Batch:
    out = ctypes.c_void_p()
    _check(_lib.flic_batch_create(max_frames, ctypes.byref(out)))
    return Batch(out.value, max_frames)


def flic_batch_destroy(b: Batch) -> None:
    b.close()


def flic_batch_set_tuning(b: Batch, px_per_cta: int = 0, threads: int = 0, max_strips: int = 0,
                          ctas_per_sm: int = 0) -> None:
    _check(_lib.flic_batch_set_tuning(b.ptr, px_per_cta, threads, max_strips, ctas_per_sm))


def flic_batch_set_schedule(b: Batch, p3_delay_waves: int = 8) -> None:
    _check(_lib.flic_batch_set_schedule(b.ptr, p3_delay_waves))


def flic_batch_last_plan(b: Batch) -> dict:
    info = np.zeros(8, np.int32)
    _check(_lib.flic_batch_last_plan(b.ptr, info.ctypes.data))
    return dict(tasks=int(info[0]), grid=int(info[1]), max_strips=int(info[2]),
                threads=int(info[3]), smem=int(info[4]), strips=int(info[5]),
                frames=int(info[6]), resident_blocks=int(info[7]))


class BatchArgs:
    """Host pointer arrays for flic_label_batch, built once and reused across calls."""

    def __init__(self, handles, ranges, labels):
        n = len(handles)
        if not (len(ranges) == len(labels) == n):
            raise ValueError("handles, ranges and labels must have the same length")
        self.n = n
        self.hs = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
        self.rs = (ctypes.c_void_p * n)(*[_dptr(r, "float32", h.npix, "range")
                                          for r, h in zip(ranges, handles)])
        self.ls = (ctypes.c_void_p * n)(*[_dptr(l, "int32", h.npix, "labels")
                                          for l, h in zip(labels, handles)])
        self._keep = (handles, ranges, labels)


def flic_label_batch(b: Batch, args: BatchArgs, stream=None) -> None:
    _check(_lib.flic_label_batch(b.ptr, args.hs, args.rs, args.ls, args.n, _stream(stream)))


def _hptr(t, dtype_name: str, numel: int, what: str) -> int:
    """Host pointer of a contiguous CPU tensor (or numpy array) of the given dtype and size."""
    if isinstance(t, np.ndarray):
        if t.dtype != np.dtype(dtype_name) or not t.flags.c_contiguous or t.size != numel:
            raise ValueError(f"{what} must be a contiguous {dtype_name} array of {numel} elements")
        return t.ctypes.data
    if t.is_cuda:
        raise ValueError(f"{what} must be in host memory")
    if str(t.dtype) != f"torch.{dtype_name}" or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{what} must be a contiguous {dtype_name} tensor of {numel} elements")
    return t.data_ptr()


def flic_label_batch_host(b: Batch, handles, host_ranges, host_labels, groups: int = 0,
                          input_ready: bool = False, stream=None) -> None:
    """Label frames held in host memory, packed back to back (frame i's rows*cols values
    right after frame i-1's): host_ranges float32, host_labels int32, both page-locked for
    the copies to overlap the labelling.  The labels are in host_labels once the work on
    `stream` has finished (e.g. after torch.cuda.synchronize()).  input_ready: the readings
    are already in host_ranges, so the call need not wait for earlier work on `stream`
    (consecutive calls overlap)."""
    n = len(handles)
    total = sum(h.npix for h in handles)
    hs = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
    _check(_lib.flic_label_batch_host(b.ptr, hs, n, _hptr(host_ranges, "float32", total, "host_ranges"),
                                      _hptr(host_labels, "int32", total, "host_labels"),
                                      int(groups), FLIC_HOST_INPUT_READY if input_ready else 0,
                                      _stream(stream)))


def flic_device_status(h: Handle, clear: bool = True) -> int:
    """FLIC_OK; FLIC_ERR_TIMEOUT when a bounded device loop gave up; FLIC_ERR_INVALID when
    flic_filter_relabel met a label outside the frame."""
    st = _lib.flic_device_status(h.ptr, 1 if clear else 0)
    if st not in (FLIC_OK, FLIC_ERR_TIMEOUT, FLIC_ERR_INVALID):
        _check(st)
    return st


def flic_set_ground(h: Handle, theta: float, mount_height: float = 0.0) -> None:
    """Ground extraction before labelling (theta in radians, <= 0: off)."""
    _check(_lib.flic_set_ground(h.ptr, float(theta), float(mount_height)))


def flic_filter_relabel(h: Handle, labels, min_size: int, num_out=None, stream=None) -> None:
    """Cluster candidates: components below min_size pixels -> -1, the rest 0..N-1."""
    _check(_lib.flic_filter_relabel(h.ptr, _dptr(labels, "int32", h.npix, "labels"),
                                    int(min_size),
                                    None if num_out is None else _dptr(num_out, "int32", 1, "num_out"),
                                    _stream(stream)))


def flic_filter_relabel_batch(b: Batch, args: BatchArgs, min_size: int, num_out=None,
                              stream=None) -> None:
    """flic_filter_relabel over the frames of args (their labels buffers) in one go."""
    _check(_lib.flic_filter_relabel_batch(
        b.ptr, args.hs, args.ls, args.n, int(min_size),
        None if num_out is None else _dptr(num_out, "int32", args.n, "num_out"),
        _stream(stream)))


def flic_label_filter_batch(b: Batch, args: BatchArgs, min_size: int, num_out=None,
                            stream=None) -> None:
    """flic_label_batch then flic_filter_relabel_batch over args, the sizes counted while
    labelling (one call; the labels buffers receive the kept components' ids or -1)."""
    _check(_lib.flic_label_filter_batch(
        b.ptr, args.hs, args.rs, args.ls, args.n, int(min_size),
        None if num_out is None else _dptr(num_out, "int32", args.n, "num_out"),
        _stream(stream)))


def flic_debug_set_iter_limit(h: Handle, limit: int) -> None:
    _check(_lib.flic_debug_set_iter_limit(h.ptr, limit))


def flic_project_noalloc(rows: int, cols: int, elevation, az_step: float, xyz, range_out,
                         point_pixel, stream=None) -> None:
    """flic_project without a handle or any allocation (static working memory in libflic)."""
    elev = np.ascontiguousarray(elevation, dtype=np.float64)
    n = xyz.numel() // 3
    _check(_lib.flic_project_noalloc(rows, cols, elev.ctypes.data, float(az_step),
                                     _dptr(xyz, "float32", 3 * n, "xyz"), n,
                                     _dptr(range_out, "float32", rows * cols, "range_out"),
                                     _dptr(point_pixel, "int32", n, "point_pixel"),
                                     _stream(stream)))


class flic_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("sensor", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("n", ctypes.c_int64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class Completion(typing.NamedTuple):
    """One completion record, copied out of the server (flic_completion's fields)."""
    tag: int
    sensor: int
    kind: int
    n: int
    status: int
    batch_size: int
    t_submit: float
    t_launch: float
    t_done: float


class Server:
    def __init__(self, ptr: int):
        self.ptr = ptr
        self._poll_buf = None

    def close(self) -> None:
        if self.ptr:
            ptr, self.ptr = self.ptr, None  # freed even when the call reports an error
            _check(_lib.flic_server_destroy(ptr))

    def __del__(self):
        try:
            if self.ptr:
                _lib.flic_server_destroy(self.ptr)
        except Exception:
            pass


def flic_server_create(sensors, max_points, nstreams: int = 2, max_batch: int = 256,
                       mem_budget: int = 1 << 30, max_queue: int = 4096) -> Server:
    n = len(sensors)
    hs = (ctypes.c_void_p * n)(*[h.ptr for h in sensors])
    mp = (ctypes.c_int64 * n)(*[int(x) for x in max_points])
    out = ctypes.c_void_p()
    _check(_lib.flic_server_create(hs, n, mp, nstreams, max_batch, int(mem_budget), max_queue,
                                   ctypes.byref(out)))
    return Server(out.value)


def flic_server_submit(srv: Server, sensor: int, kind: int, host_in, host_out, tag: int) -> int:
    """host_in/host_out: pinned CPU tensors (float32 input, int32 output).  Returns the
    status (FLIC_OK or FLIC_ERR_BUSY when the admission queue is full)."""
    n = host_in.numel() // 3 if kind == 1 else host_in.numel()
    st = _lib.flic_server_submit(srv.ptr, sensor, kind, host_in.data_ptr(), n,
                                 host_out.data_ptr(), tag)
    if st not in (FLIC_OK, FLIC_ERR_BUSY):
        _check(st)
    return st


def flic_server_hold(srv: Server, hold: bool) -> None:
    _check(_lib.flic_server_hold(srv.ptr, 1 if hold else 0))


def flic_server_poll(srv: Server, max_records: int = 4096):
    """Completion records since the last poll (at most max_records), as Completion tuples.
    The records are copied out of one receive buffer that the Server keeps, so a caller
    that holds many records holds no ctypes buffers (a fresh 229 KB buffer per poll, kept
    alive by every record taken from it, grew the process by hundreds of MB per second of
    high-rate serving)."""
    if srv._poll_buf is None or len(srv._poll_buf[0]) < max_records:
        buf = (flic_completion * max_records)()
        srv._poll_buf = (buf, np.ctypeslib.as_array(buf))
    buf, view = srv._poll_buf
    k = _lib.flic_server_poll(srv.ptr, buf, max_records)
    return [Completion._make(t) for t in view[:k].tolist()]


def flic_server_drain(srv: Server, timeout_s: float = 30.0) -> None:
    _check(_lib.flic_server_drain(srv.ptr, float(timeout_s)))


def flic_server_stats(srv: Server) -> dict:
    out = (ctypes.c_int64 * 8)()
    _check(_lib.flic_server_stats(srv.ptr, out))
    keys = ["submitted", "rejected", "completed", "batches", "largest_batch", "slots",
            "slot_bytes", "in_flight"]
    return dict(zip(keys, [int(x) for x in out]))


def flic_server_destroy(srv: Server) -> None:
    srv.close()


def flic_server_clock() -> float:
    return _lib.flic_server_clock()
