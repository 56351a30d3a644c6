"""CPU oracle of the FLIC hot path (arXiv 2003.00575) — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  The product path (``paper_2003_00575_gb300``) never imports it and shares
no code with it.  The arithmetic lives in ``flic_oracle.c`` (plain C, fp32 without
contraction, fp64 where stated); this module compiles it with gcc and exposes it through
ctypes with numpy arrays.

Functions and the passages they follow:
  tables      Eq. 3 constants per row and offset (§III-B, §III-B-2); optionally the
              true angle between the rays of a row (exact_ray)
  pred        Eq. 2/3 squared distance against delta (§III-B)
  edges       per-pixel edge bits for offsets 1..S (§III-B-1 binary images, §III-B-2)
  label       BFS connected-component labelling, min-index labels (§III-B-1); with
              diagonal=True also the diagonal Map Connections (§III-B-2)
  tables_diag Eq. 3 constants of the diagonal pairs (r, c)-(r+k, c+-k): the squared distance
              of the two unit rays, in double
  flips       FP64 Eq. 2 decision vs the fp32 one
  project     spherical projection of xyz into the range image (§I)
  scatter     labels back to points (§I, Fig. 1)
  ground      ground extraction by the angle to the reading above (§III-A, Eq. 1)
  label_ground  labelling with the ground removed first (§III-A before §III-B)
  filter_relabel  cluster candidates: components below a minimum size dropped, the rest
              numbered by their minimum index (§III-B, the minimum of 100 points)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_flic_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile flic_oracle.c into an in-tree shared object (gcc, a second or two)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        lib.oracle_tables.argtypes = [i32, P, f64, i32, P, P]
        lib.oracle_tables.restype = None
        lib.oracle_tables_ex.argtypes = [i32, P, f64, i32, i32, P, P]
        lib.oracle_tables_ex.restype = None
        lib.oracle_pred.argtypes = [f32, f32, f32, f32]
        lib.oracle_pred.restype = i32
        lib.oracle_pred_paper_form.argtypes = [f32, f32, f32, f32]
        lib.oracle_pred_paper_form.restype = i32
        lib.oracle_edges.argtypes = [i32, i32, P, P, P, i32, f32, i32, P]
        lib.oracle_edges_ex.argtypes = [i32, i32, P, P, P, i32, f32, i32, i32, P]
        lib.oracle_edges_ex.restype = None
        lib.oracle_edges.restype = None
        lib.oracle_label.argtypes = [i32, i32, P, P, P, i32, f32, i32, P]
        lib.oracle_label_ex.argtypes = [i32, i32, P, P, P, i32, f32, i32, i32, P]
        lib.oracle_label_ex.restype = i64
        lib.oracle_label.restype = i64
        lib.oracle_flips.argtypes = [i32, i32, P, P, f64, P, P, i32, f32, i32, P, P]
        lib.oracle_flips.restype = None
        lib.oracle_flips_paper_form.argtypes = [i32, i32, P, P, f64, i32, f32, i32, P, P]
        lib.oracle_flips_paper_form.restype = None
        lib.oracle_proj_tables.argtypes = [i32, i32, P, f64, P, P, P]
        lib.oracle_proj_tables.restype = i32
        lib.oracle_project.argtypes = [i32, i32, P, f64, P, i64, P, P, P]
        lib.oracle_project.restype = i32
        lib.oracle_scatter.argtypes = [P, P, i64, P]
        lib.oracle_scatter.restype = None
        lib.oracle_ground.argtypes = [i32, i32, P, P, f64, f64, P]
        lib.oracle_ground.restype = None
        lib.oracle_tables_diag.argtypes = [i32, P, f64, i32, P]
        lib.oracle_tables_diag.restype = None
        lib.oracle_label_diag.argtypes = [i32, i32, P, P, P, P, i32, f32, i32, P]
        lib.oracle_label_diag.restype = i64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def tables(elevation, az_step: float, skip: int, exact_ray: bool = False):
    """(Kv, Kh), each float32 [rows, skip]: 4 sin^2(alpha/2) per row and offset (Eq. 3).
    exact_ray: the horizontal alpha is the true angle between the rays of a row k columns
    apart (K = 4 cos^2(e) sin^2(k step / 2)) instead of k times the azimuth step."""
    elev = _f64(elevation)
    R = elev.shape[0]
    kv = np.zeros((R, skip), np.float32)
    kh = np.zeros((R, skip), np.float32)
    _load().oracle_tables_ex(R, _ptr(elev), float(az_step), skip, int(bool(exact_ray)),
                             _ptr(kv), _ptr(kh))
    return kv, kh


def pred(a: float, b: float, K: float, delta: float) -> bool:
    """fp32 edge decision for one pair: (a-b)^2 + K*(a*b) <= delta^2 (Eq. 2/3)."""
    d = np.float32(delta)
    return bool(_load().oracle_pred(float(np.float32(a)), float(np.float32(b)),
                                    float(np.float32(K)), float(d * d)))


def pred_paper_form(a: float, b: float, C2: float, delta: float) -> bool:
    """fp32 decision in the literal Eq. 3 form a*a + b*b - C2*(a*b) <= delta^2."""
    d = np.float32(delta)
    return bool(_load().oracle_pred_paper_form(float(np.float32(a)), float(np.float32(b)),
                                               float(np.float32(C2)), float(d * d)))


def edges(range_img, elevation, az_step: float, delta: float, skip: int, wrap: bool = True,
          exact_ray: bool = False, lattice: bool = False):
    """uint16 [rows, cols] edge bits: bit k-1 horizontal (+k, wrap), bit 8+k-1 vertical (+k).
    lattice: the sparse Map Connection (§III-B-2), offset 1 from every pixel and offset S
    only from pixels whose row and column are multiples of S."""
    rng = _f32(range_img)
    R, C = rng.shape
    kv, kh = tables(elevation, az_step, skip, exact_ray)
    mask = np.zeros((R, C), np.uint16)
    _load().oracle_edges_ex(R, C, _ptr(rng), _ptr(kv), _ptr(kh), skip, float(np.float32(delta)),
                            int(bool(wrap)), int(bool(lattice)), _ptr(mask))
    return mask


def tables_diag(elevation, az_step: float, skip: int):
    """Kd float32 [rows, skip]: Eq. 3's constant of the diagonal pair (r, c)-(r+k, c+-k),
    2 - 2 cos(alpha) with alpha the angle between the two beams' rays (0 where r+k >= rows)."""
    elev = _f64(elevation)
    R = elev.shape[0]
    kd = np.zeros((R, skip), np.float32)
    _load().oracle_tables_diag(R, _ptr(elev), float(az_step), skip, _ptr(kd))
    return kd


def label(range_img, elevation, az_step: float, delta: float, skip: int, wrap: bool = True,
          exact_ray: bool = False, lattice: bool = False, diagonal: bool = False):
    """int32 [rows, cols] labels: min linear index of the component, -1 for invalid.
    lattice: the sparse Map Connection of §III-B-2 (see edges); diagonal: the diagonal Map
    Connections (r, c)-(r+k, c+-k), k = 1..skip, as well (not with lattice)."""
    rng = _f32(range_img)
    R, C = rng.shape
    kv, kh = tables(elevation, az_step, skip, exact_ray)
    out = np.empty((R, C), np.int32)
    if diagonal:
        if lattice:
            raise ValueError("diagonal Map Connections are not combined with the sparse map")
        kd = tables_diag(elevation, az_step, skip)
        n = _load().oracle_label_diag(R, C, _ptr(rng), _ptr(kv), _ptr(kh), _ptr(kd), skip,
                                      float(np.float32(delta)), int(bool(wrap)), _ptr(out))
    else:
        n = _load().oracle_label_ex(R, C, _ptr(rng), _ptr(kv), _ptr(kh), skip,
                                    float(np.float32(delta)), int(bool(wrap)),
                                    int(bool(lattice)), _ptr(out))
    if n < 0:
        raise MemoryError("oracle_label: out of memory")
    return out


def flips(range_img, elevation, az_step: float, delta: float, skip: int, wrap: bool = True):
    """(candidate_pairs, fp64_flips, max |D - delta| over flips) for one frame."""
    rng = _f32(range_img)
    R, C = rng.shape
    elev = _f64(elevation)
    kv, kh = tables(elev, az_step, skip)
    out = np.zeros(2, np.int64)
    dev = np.zeros(1, np.float64)
    _load().oracle_flips(R, C, _ptr(rng), _ptr(elev), float(az_step), _ptr(kv), _ptr(kh), skip,
                         float(np.float32(delta)), int(bool(wrap)), _ptr(out), _ptr(dev))
    return int(out[0]), int(out[1]), float(dev[0])


def flips_paper_form(range_img, elevation, az_step: float, delta: float, skip: int,
                     wrap: bool = True):
    """(candidate_pairs, flips, flips with |D - delta| >= 1e-5 m, max |D - delta|) of the
    literal Eq. 3 form d1*d1 + d2*d2 - (2 cos alpha)*d1*d2 against the double-precision
    Eq. 2, for one frame (a diagnostic of the cancellation the main form avoids)."""
    rng = _f32(range_img)
    R, C = rng.shape
    out = np.zeros(3, np.int64)
    dev = np.zeros(1, np.float64)
    _load().oracle_flips_paper_form(R, C, _ptr(rng), _ptr(_f64(elevation)), float(az_step), skip,
                                    float(np.float32(delta)), int(bool(wrap)), _ptr(out),
                                    _ptr(dev))
    return int(out[0]), int(out[1]), int(out[2]), float(dev[0])


def proj_tables(rows: int, cols: int, elevation, az_step: float):
    """(colb [cols,2], rowb [rows+1,2], sorted_row [rows]) boundary tables of the projection."""
    elev = _f64(elevation)
    colb = np.zeros((cols, 2), np.float32)
    rowb = np.zeros((rows + 1, 2), np.float32)
    srow = np.zeros(rows, np.int32)
    rc = _load().oracle_proj_tables(rows, cols, _ptr(elev), float(az_step), _ptr(colb),
                                    _ptr(rowb), _ptr(srow))
    if rc != 0:
        raise ValueError("projection needs >= 2 rows with distinct elevations")
    return colb, rowb, srow


def project(xyz, rows: int, cols: int, elevation, az_step: float):
    """(range_img float32 [rows,cols], point_pixel int32 [n], winner int32 [rows*cols])."""
    pts = _f32(xyz).reshape(-1, 3)
    n = pts.shape[0]
    elev = _f64(elevation)
    rimg = np.zeros((rows, cols), np.float32)
    pix = np.zeros(n, np.int32)
    win = np.zeros(rows * cols, np.int32)
    rc = _load().oracle_project(rows, cols, _ptr(elev), float(az_step), _ptr(pts), n,
                                _ptr(rimg), _ptr(pix), _ptr(win))
    if rc != 0:
        raise ValueError("oracle_project: bad projection tables or out of memory")
    return rimg, pix, win


def scatter(labels, point_pixel):
    """int32 [n]: labels[point_pixel[i]] or -1."""
    lab = np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)
    pix = np.ascontiguousarray(point_pixel, dtype=np.int32)
    out = np.empty(pix.shape[0], np.int32)
    _load().oracle_scatter(_ptr(lab), _ptr(pix), pix.shape[0], _ptr(out))
    return out


def filter_relabel(labels, min_size: int):
    """Cluster candidates (§III-B: labelled clusters with fewer than a minimum number of
    measurements are discarded as noise; the paper uses 100).  ``labels`` is the output of
    ``label`` (each measurement carries the minimum index of its component, -1 elsewhere).
    Components with fewer than ``min_size`` pixels are dropped (their pixels become -1);
    the others are numbered 0..N-1 in ascending order of their minimum index, i.e. in the
    raster order of their first pixel.  Returns (int32 labels of the same shape, N).

    The plain definition: a histogram of the labels (np.bincount), the kept minima in
    ascending order (np.flatnonzero), each pixel mapped to the rank of its minimum."""
    lab = np.asarray(labels).astype(np.int64)
    flat = lab.reshape(-1)
    out = np.full(flat.shape, -1, np.int32)
    v = flat >= 0
    if not v.any():
        return out.reshape(lab.shape), 0
    counts = np.bincount(flat[v], minlength=flat.size)
    kept = np.flatnonzero((counts > 0) & (counts >= min_size))
    ids = np.full(flat.size, -1, np.int64)
    ids[kept] = np.arange(kept.size)
    out[v] = ids[flat[v]]
    return out.reshape(lab.shape), int(kept.size)


def ground(range_img, elevation, theta: float, mount_height: float = 0.0):
    """bool [rows, cols]: the readings §III-A removes as ground — spanning a horizontal
    surface with the reading above (Eq. 1, tangent form; +-theta radians), the first row
    deciding as the second; with mount_height > 0, horizontal readings above the line
    z = rho tan(theta) - mount_height are kept (not ground)."""
    rng = _f32(range_img)
    R, C = rng.shape
    elev = _f64(elevation)
    mask = np.zeros((R, C), np.uint8)
    _load().oracle_ground(R, C, _ptr(rng), _ptr(elev), float(theta), float(mount_height),
                          _ptr(mask))
    return mask.astype(bool)


def label_ground(range_img, elevation, az_step: float, delta: float, skip: int, wrap: bool,
                 theta: float, mount_height: float = 0.0):
    """Labels with the ground removed first: ground readings become non-measurements."""
    rng = _f32(range_img)
    g = ground(rng, elevation, theta, mount_height)
    return label(np.where(g, np.float32(0), rng), elevation, az_step, delta, skip, wrap)
