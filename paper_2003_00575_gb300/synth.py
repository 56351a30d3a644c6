"""Seeded synthetic lidar frames (inputs only; none of the method's arithmetic lives here).

A ray caster from the sensor origin stands in for the paper's datasets (a 64-beam
Velodyne log and SemanticKITTI, §IV), which are not available here.  Each frame is a
range image (row = beam, row 0 the top beam; column = azimuth bin) of hits on a ground
plane z = -1.7 m (cut off at 120 m, the reliable range quoted in §III-B) and on
axis-aligned boxes and vertical cylinders, with Gaussian range noise and dropouts
(range 0 = no return).  The ground is kept, so one large component spans every frame.

Both the CUDA path (through its tests and the bench) and the CPU oracle are fed from
these generators; this module imports neither of them.

Configurations (sizes in pixels):
  c1  16 x 1800, +-15 deg, 0.2 deg step, 20 boxes, sigma 0.02, 5 % dropout, delta 0.5, S 1
  c2  64 x 2048, +-22.5 deg, 60 boxes + 30 cylinders, sigma 0.02, 5 % dropout, delta 0.5, S 3
  c3  128 x 2048, +-22.5 deg, 80 poles at 2-10 m in front of 100 boxes, 20 % dropout plus
      500 dropout blocks of 1-8 px, sigma 0.03, delta 0.4, S 5; plus one xyz point per pixel
  c4  256 frames, shapes uniform over {16x1800, 32x1024, 64x2048, 128x2048}, per-frame
      elevation jitter U(+-0.05 deg), delta U(0.3, 0.6), S U{1..5}, c2-style scenes
  c5  4 sensors with the c4 shapes; frames as range images or xyz clouds of 30k-260k points
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GROUND_Z = -1.7
MAX_RANGE = 120.0

# (rows, cols, lower elevation deg, upper elevation deg) of the four sensor shapes
SHAPES = [(16, 1800, -15.0, 15.0), (32, 1024, -20.0, 20.0), (64, 2048, -22.5, 22.5),
          (128, 2048, -22.5, 22.5)]


@dataclass
class Sensor:
    rows: int
    cols: int
    elevation: np.ndarray  # float64 [rows], radians, row 0 = top beam
    az_step: float         # radians per column


@dataclass
class Frame:
    sensor: Sensor
    range: np.ndarray        # float32 [rows, cols]; 0 = no return
    delta: float
    skip: int
    object_id: np.ndarray    # int32 [rows, cols]; -1 no hit, 0 ground, 1.. objects
    xyz: np.ndarray | None = None   # float32 [n, 3] when the frame comes as a point cloud
    name: str = ""
    meta: dict = field(default_factory=dict)


def make_sensor(rows: int, cols: int, lo_deg: float, hi_deg: float,
                jitter_deg: float = 0.0, rng: np.random.Generator | None = None) -> Sensor:
    """Beams uniformly spaced from hi (row 0) down to lo, plus sorted U(+-jitter) offsets."""
    if rows > 1:
        e = hi_deg - np.arange(rows) * (hi_deg - lo_deg) / (rows - 1)
    else:
        e = np.array([0.5 * (hi_deg + lo_deg)])
    if jitter_deg > 0.0:
        assert rng is not None
        j = np.sort(rng.uniform(-jitter_deg, jitter_deg, rows))[::-1]
        e = e + j
    return Sensor(rows, cols, np.radians(e).astype(np.float64), 2.0 * math.pi / cols)


def ray_dirs(sensor: Sensor):
    """Unit ray directions at the pixel centres: (dx, dy, dz), each float64 [rows, cols]."""
    el = sensor.elevation[:, None]
    az = (np.arange(sensor.cols) + 0.5)[None, :] * sensor.az_step
    ce = np.cos(el)
    return ce * np.cos(az), ce * np.sin(az), np.sin(el) * np.ones_like(az)


@dataclass
class Box:
    x0: float
    x1: float
    y0: float
    y1: float
    z0: float
    z1: float


@dataclass
class Cylinder:
    cx: float
    cy: float
    r: float
    z0: float
    z1: float


def _cols_for(sensor: Sensor, cx: float, cy: float, rb: float) -> np.ndarray:
    """Column indices whose rays can reach an object bounded by a circle (cx, cy, rb)."""
    d = math.hypot(cx, cy)
    C = sensor.cols
    if d <= rb + 1e-6:
        return np.arange(C)
    w = math.asin(min(1.0, rb / d))
    phi = math.atan2(cy, cx) % (2.0 * math.pi)
    c_lo = int(math.floor((phi - w) / sensor.az_step)) - 1
    c_hi = int(math.ceil((phi + w) / sensor.az_step)) + 1
    if c_hi - c_lo + 1 >= C:
        return np.arange(C)
    return np.arange(c_lo, c_hi + 1) % C


def _hit_box(b: Box, dx, dy, dz):
    """Entry distance of rays from the origin into the box (inf where missed)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t_lo = np.full(dx.shape, -np.inf)
        t_hi = np.full(dx.shape, np.inf)
        for d, lo, hi in ((dx, b.x0, b.x1), (dy, b.y0, b.y1), (dz, b.z0, b.z1)):
            inv = 1.0 / d
            t1 = lo * inv
            t2 = hi * inv
            tmin = np.minimum(t1, t2)
            tmax = np.maximum(t1, t2)
            par = d == 0.0
            inside = (lo <= 0.0) & (0.0 <= hi)
            tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
            tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
            t_lo = np.maximum(t_lo, tmin)
            t_hi = np.minimum(t_hi, tmax)
        hit = (t_lo <= t_hi) & (t_lo > 0.0)
        return np.where(hit, t_lo, np.inf)


def _hit_cylinder(cy_: Cylinder, dx, dy, dz):
    """Nearest hit of rays from the origin with a closed vertical cylinder (inf if none)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        a = dx * dx + dy * dy
        b = -2.0 * (dx * cy_.cx + dy * cy_.cy)
        c = cy_.cx ** 2 + cy_.cy ** 2 - cy_.r ** 2
        disc = b * b - 4.0 * a * c
        sq = np.sqrt(np.maximum(disc, 0.0))
        t_side = (-b - sq) / (2.0 * a)
        z = t_side * dz
        side_ok = (disc >= 0.0) & (t_side > 0.0) & (z >= cy_.z0) & (z <= cy_.z1)
        best = np.where(side_ok, t_side, np.inf)
        for zc in (cy_.z0, cy_.z1):
            tc = zc / dz
            px = tc * dx - cy_.cx
            py = tc * dy - cy_.cy
            cap_ok = (tc > 0.0) & (px * px + py * py <= cy_.r ** 2)
            best = np.minimum(best, np.where(cap_ok, tc, np.inf))
        return best


def raycast(sensor: Sensor, boxes, cylinders):
    """Nearest-hit range (float64, 0 = none) and object id (-1 none, 0 ground, 1.. objects)."""
    dx, dy, dz = ray_dirs(sensor)
    R, C = sensor.rows, sensor.cols
    with np.errstate(divide="ignore"):
        t_ground = np.where(dz < 0.0, GROUND_Z / dz, np.inf)
    t_ground = np.where(t_ground <= MAX_RANGE, t_ground, np.inf)
    best = t_ground.copy()
    oid = np.where(np.isfinite(best), 0, -1).astype(np.int32)
    objs = [(b, _hit_box, 0.5 * (b.x0 + b.x1), 0.5 * (b.y0 + b.y1),
             0.5 * math.hypot(b.x1 - b.x0, b.y1 - b.y0)) for b in boxes]
    objs += [(c, _hit_cylinder, c.cx, c.cy, c.r) for c in cylinders]
    for i, (o, fn, cx, cy, rb) in enumerate(objs):
        cols = _cols_for(sensor, cx, cy, rb)
        t = fn(o, dx[:, cols], dy[:, cols], dz[:, cols])
        cur = best[:, cols]
        closer = t < cur
        if closer.any():
            best[:, cols] = np.where(closer, t, cur)
            oid[:, cols] = np.where(closer, i + 1, oid[:, cols])
    rng = np.where(np.isfinite(best) & (best <= MAX_RANGE), best, 0.0)
    oid = np.where(rng > 0.0, oid, -1).astype(np.int32)
    return rng, oid


def _place(g: np.random.Generator, r_lo: float, r_hi: float):
    d = g.uniform(r_lo, r_hi)
    a = g.uniform(0.0, 2.0 * math.pi)
    return d * math.cos(a), d * math.sin(a)


def random_boxes(g: np.random.Generator, n: int, r_lo: float, r_hi: float,
                 side_lo: float = 0.5, side_hi: float = 5.0):
    """n boxes resting on the ground, sides U(side_lo, side_hi), centres at radius
    U(r_lo, r_hi); a box whose footprint comes within 0.5 m of the sensor is redrawn."""
    out = []
    while len(out) < n:
        cx, cy = _place(g, r_lo, r_hi)
        sx, sy, sz = g.uniform(side_lo, side_hi, 3)
        b = Box(cx - sx / 2, cx + sx / 2, cy - sy / 2, cy + sy / 2, GROUND_Z, GROUND_Z + sz)
        if b.x0 - 0.5 < 0.0 < b.x1 + 0.5 and b.y0 - 0.5 < 0.0 < b.y1 + 0.5:
            continue
        out.append(b)
    return out


def random_cylinders(g: np.random.Generator, n: int, r_lo: float, r_hi: float,
                     rad_lo: float, rad_hi: float, h_lo: float, h_hi: float):
    out = []
    for _ in range(n):
        cx, cy = _place(g, r_lo, r_hi)
        rad = g.uniform(rad_lo, rad_hi)
        h = g.uniform(h_lo, h_hi)
        out.append(Cylinder(cx, cy, rad, GROUND_Z, GROUND_Z + h))
    return out


def finish(g: np.random.Generator, rng64: np.ndarray, sigma: float, dropout: float,
           blocks: int = 0) -> np.ndarray:
    """Gaussian noise on hits (clamped positive), i.i.d. dropout, rectangular dropout blocks."""
    R, C = rng64.shape
    hit = rng64 > 0.0
    noisy = rng64 + g.normal(0.0, sigma, rng64.shape)
    noisy = np.where(hit, np.maximum(noisy, 1e-3), 0.0)
    drop = g.random(rng64.shape) < dropout
    noisy = np.where(drop, 0.0, noisy)
    for _ in range(blocks):
        h, w = g.integers(1, 9, 2)
        r0 = g.integers(0, R)
        c0 = g.integers(0, C)
        rows = np.arange(r0, min(R, r0 + h))
        cols = np.arange(c0, c0 + w) % C
        noisy[np.ix_(rows, cols)] = 0.0
    return noisy.astype(np.float32)


def pixel_cloud(g: np.random.Generator, sensor: Sensor, rimg: np.ndarray,
                pixels: np.ndarray | None = None, jitter: float = 0.25) -> np.ndarray:
    """xyz points along pixel-centre rays at each pixel's range, with U(+-jitter bin)
    angular jitter.  pixels = flat indices to emit (default: every pixel, in order);
    invalid pixels give the origin."""
    R, C = rimg.shape
    if pixels is None:
        pixels = np.arange(R * C)
    r = pixels // C
    c = pixels % C
    el = sensor.elevation
    # row spacing at each beam (one-sided at the ends)
    sp = np.abs(np.gradient(el)) if R > 1 else np.array([0.01])
    e = el[r] + g.uniform(-jitter, jitter, r.shape) * sp[r]
    a = (c + 0.5 + g.uniform(-jitter, jitter, c.shape)) * sensor.az_step
    d = rimg.reshape(-1)[pixels].astype(np.float64)
    ce = np.cos(e)
    xyz = np.stack([d * ce * np.cos(a), d * ce * np.sin(a), d * np.sin(e)], axis=1)
    return xyz.astype(np.float32)


def config_c1(seed: int = 1) -> Frame:
    g = np.random.Generator(np.random.PCG64(seed))
    s = make_sensor(16, 1800, -15.0, 15.0)
    rng64, oid = raycast(s, random_boxes(g, 20, 3.0, 40.0), [])
    return Frame(s, finish(g, rng64, 0.02, 0.05), 0.5, 1, oid, name="c1 16x1800 S1")


def _c2_scene(g: np.random.Generator, s: Sensor):
    boxes = random_boxes(g, 60, 3.0, 40.0)
    cyls = random_cylinders(g, 30, 3.0, 40.0, 0.05, 0.5, 1.0, 4.0)
    return raycast(s, boxes, cyls)


def config_c2(seed: int = 2) -> Frame:
    g = np.random.Generator(np.random.PCG64(seed))
    s = make_sensor(64, 2048, -22.5, 22.5)
    rng64, oid = _c2_scene(g, s)
    return Frame(s, finish(g, rng64, 0.02, 0.05), 0.5, 3, oid, name="c2 64x2048 S3")


def config_c3(seed: int = 3, with_xyz: bool = True) -> Frame:
    g = np.random.Generator(np.random.PCG64(seed))
    s = make_sensor(128, 2048, -22.5, 22.5)
    poles = random_cylinders(g, 80, 2.0, 10.0, 0.05, 0.15, 3.0, 3.0)
    boxes = random_boxes(g, 100, 12.0, 40.0)
    rng64, oid = raycast(s, boxes, poles)
    rimg = finish(g, rng64, 0.03, 0.20, blocks=500)
    f = Frame(s, rimg, 0.4, 5, oid, name="c3 128x2048 S5")
    if with_xyz:
        f.xyz = pixel_cloud(g, s, rimg)
    return f


def config_c4_frame(seed: int) -> Frame:
    g = np.random.Generator(np.random.PCG64(seed))
    R, C, lo, hi = SHAPES[int(g.integers(0, 4))]
    s = make_sensor(R, C, lo, hi, jitter_deg=0.05, rng=g)
    delta = float(np.float32(g.uniform(0.3, 0.6)))
    skip = int(g.integers(1, 6))
    rng64, oid = _c2_scene(g, s)
    return Frame(s, finish(g, rng64, 0.02, 0.05), delta, skip, oid,
                 name=f"c4 seed{seed} {R}x{C} S{skip}")


def config_c4(n: int = 256, first_seed: int = 100):
    """The batch: frames with seeds first_seed .. first_seed + n - 1."""
    return [config_c4_frame(first_seed + i) for i in range(n)]


def c5_sensors():
    """The four serving sensors (fixed tables), one per c4 shape."""
    return [make_sensor(R, C, lo, hi) for (R, C, lo, hi) in SHAPES]


def c5_frame(sensor: Sensor, seed: int, as_cloud: bool) -> Frame:
    """One served frame: a c2-style scene; as a cloud of U(30k, 260k) points drawn from
    the valid pixels with replacement (so several points may share a pixel)."""
    g = np.random.Generator(np.random.PCG64(seed))
    rng64, oid = _c2_scene(g, sensor)
    rimg = finish(g, rng64, 0.02, 0.05)
    f = Frame(sensor, rimg, 0.5, 3, oid, name=f"c5 {sensor.rows}x{sensor.cols}")
    if as_cloud:
        n = int(g.integers(30_000, 260_001))
        valid = np.flatnonzero(rimg.reshape(-1) > 0)
        pix = g.choice(valid, size=n, replace=True)
        f.xyz = pixel_cloud(g, sensor, rimg, pixels=pix)
    return f
