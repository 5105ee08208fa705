"""Seeded synthetic depth + colour frames for hash-blocked TSDF fusion.

This module is the only code shared by the CUDA path's callers and the CPU
oracle's callers: it produces *inputs* (depth images, 8-bit colour, pinhole
intrinsics, camera-to-world poses) and holds none of the fusion arithmetic.
The geometry is analytic ray casting in float64; results are stored in the
frame's types (float32 depth, uint8 RGB, float32 intrinsics and pose).

Randomness is counter based, so every pixel's noise is a pure function of
(seed, stream, index) and identical on every machine:
  splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) mixes a 64-bit counter; the top 53 bits give a
  uniform double in [0, 1); Box-Muller gives a standard normal.

Scenes (stand-ins for the paper's sphere/plane cells and TartanAir rooms,
Section 5 and Table "cells"; the real data is not available here):
  * ``plane_sphere``: camera 1.5 m from a fronto-parallel plane with a 0.3 m
    sphere centred 1.0 m in front of the camera (160x120, fx=fy=140).
  * ``room``: axis-aligned 6.4 x 2.7 x 6.4 m room (floor, ceiling, four walls)
    with seeded boxes and spheres, depths 0.5-4 m (640x480, fx=fy=525,
    cx=319.5, cy=239.5), seen from an orbit of radius 0.8 m around the room
    centre whose pitch sweeps +-26 deg three times, so a full orbit sees the
    floor and ceiling too.
Depth noise follows the Kinect axial model of Nguyen, Izadi and Lovell
(3DIMPVT 2012): sigma(z) = 0.0012 + 0.0019 (z - 0.4)^2 metres, Gaussian per
pixel, followed by 5 % i.i.d. dropout to 0 (invalid).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_U64 = np.uint64
_GOLD = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied element-wise to a uint64 array (wraps mod 2^64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLD
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def _stream_base(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed & 0xFFFFFFFF) << 20 ^ (stream & 0xFFFFF)], dtype=np.uint64)
    return splitmix64(splitmix64(s))[0]


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from counter stream (seed, stream)."""
    base = _stream_base(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(n, dtype=np.uint64) + base
    u = splitmix64(ctr) >> _U64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on two counter streams)."""
    u1 = uniform(seed, 2 * stream + 1, n)
    u2 = uniform(seed, 2 * stream + 2, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Analytic primitives (float64 ray casting)
# ----------------------------------------------------------------------------
@dataclass
class Plane:
    n: tuple  # unit normal
    c: float  # n . x = c
    albedo: tuple = (180, 180, 180)


@dataclass
class Sphere:
    centre: tuple
    r: float
    albedo: tuple = (200, 60, 60)


@dataclass
class Box:
    lo: tuple
    hi: tuple
    albedo: tuple = (60, 120, 200)


def _hit_plane(o, d, p: Plane):
    n = np.asarray(p.n, dtype=np.float64)
    den = d @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = (p.c - o @ n) / den
    lam = np.where(np.abs(den) > 1e-12, lam, np.inf)
    return np.where(lam > 1e-9, lam, np.inf)


def _hit_sphere(o, d, s: Sphere):
    oc = o - np.asarray(s.centre, dtype=np.float64)
    a = np.einsum("ij,ij->i", d, d)
    b = np.einsum("ij,ij->i", d, oc)
    c = np.einsum("ij,ij->i", oc, oc) - s.r * s.r
    disc = b * b - a * c
    sq = np.sqrt(np.maximum(disc, 0.0))
    l0 = (-b - sq) / a
    l1 = (-b + sq) / a
    lam = np.where(l0 > 1e-9, l0, np.where(l1 > 1e-9, l1, np.inf))
    return np.where(disc >= 0.0, lam, np.inf)


def _hit_box(o, d, bx: Box):
    lo = np.asarray(bx.lo, dtype=np.float64)
    hi = np.asarray(bx.hi, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    lam = np.where(tmin > 1e-9, tmin, tmax)
    ok = (tmax >= np.maximum(tmin, 1e-9))
    return np.where(ok, lam, np.inf)


def raycast(width, height, intr, pose, prims):
    """Camera-z depth (float64, inf where nothing is hit) and primitive id per pixel.

    Pixel (u, v) is the pixel centre (integer coordinates); its camera-frame ray
    is ((u - cx)/fx, (v - cy)/fy, 1), so the hit parameter equals camera z.
    """
    fx, fy, cx, cy = (float(x) for x in intr)
    vv, uu = np.mgrid[0:height, 0:width]
    dc = np.stack([(uu.ravel() - cx) / fx, (vv.ravel() - cy) / fy,
                   np.ones(width * height)], axis=1)
    pose = np.asarray(pose, dtype=np.float64)
    R, t = pose[:3, :3], pose[:3, 3]
    dw = dc @ R.T
    o = np.broadcast_to(t, dw.shape)
    best = np.full(width * height, np.inf)
    ident = np.full(width * height, -1, dtype=np.int64)
    for i, p in enumerate(prims):
        if isinstance(p, Plane):
            lam = _hit_plane(o, dw, p)
        elif isinstance(p, Sphere):
            lam = _hit_sphere(o, dw, p)
        else:
            lam = _hit_box(o, dw, p)
        closer = lam < best
        best = np.where(closer, lam, best)
        ident = np.where(closer, i, ident)
    return best.reshape(height, width), ident.reshape(height, width)


# ----------------------------------------------------------------------------
# Frames
# ----------------------------------------------------------------------------
@dataclass
class Frame:
    depth: np.ndarray          # (H, W) float32, 0 = invalid
    rgb: np.ndarray            # (H, W, 3) uint8
    intr: np.ndarray           # (4,) float32: fx, fy, cx, cy
    pose: np.ndarray           # (4, 4) float32 camera-to-world, row-major
    meta: dict = field(default_factory=dict)

    @property
    def width(self) -> int:
        return int(self.depth.shape[1])

    @property
    def height(self) -> int:
        return int(self.depth.shape[0])

    @property
    def valid_points(self) -> int:
        d = self.depth
        return int(np.count_nonzero(np.isfinite(d) & (d > 0)))


def kinect_sigma(z):
    """Axial noise sigma(z) in metres (Nguyen et al. 2012)."""
    return 0.0012 + 0.0019 * (z - 0.4) ** 2


def render(width, height, intr, pose, prims, seed, noise=True, dropout=0.05,
           colour_jitter=12):
    """Ray-cast a frame, then add seeded Kinect noise, dropout and colour jitter."""
    intr32 = np.asarray(intr, dtype=np.float32)
    pose32 = np.asarray(pose, dtype=np.float32)
    z, ident = raycast(width, height, intr32.astype(np.float64),
                       pose32.astype(np.float64), prims)
    n = width * height
    hit = np.isfinite(z)
    zz = np.where(hit, z, 0.0)
    if noise:
        zz = zz + kinect_sigma(zz) * normal(seed, 1, n).reshape(height, width)
    if dropout > 0:
        drop = uniform(seed, 7, n).reshape(height, width) < dropout
        zz = np.where(drop, 0.0, zz)
    zz = np.where(hit & (zz > 0), zz, 0.0)
    depth = zz.astype(np.float32)
    alb = np.array([p.albedo for p in prims] + [(0, 0, 0)], dtype=np.int64)
    rgb = alb[ident]  # ident -1 -> last row (black)
    if colour_jitter:
        j = np.floor(uniform(seed, 11, n * 3) * (2 * colour_jitter + 1)).astype(np.int64)
        rgb = rgb + (j - colour_jitter).reshape(height, width, 3)
    rgb = np.clip(rgb, 0, 255).astype(np.uint8)
    return Frame(depth=depth, rgb=np.ascontiguousarray(rgb), intr=intr32,
                 pose=np.ascontiguousarray(pose32))


def rotation(yaw=0.0, pitch=0.0, roll=0.0):
    """Camera-to-world rotation Ry(yaw) Rx(pitch) Rz(roll); camera x right, y down, z forward."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Ry = np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    Rz = np.array([[cr, -sr, 0], [sr, cr, 0], [0, 0, 1]])
    return Ry @ Rx @ Rz


def make_pose(R, t):
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = t
    return P


# --- scene 1: plane + sphere -------------------------------------------------
PLANE_SPHERE_INTR = (140.0, 140.0, 80.0, 60.0)


def plane_sphere_prims(plane_z=1.5, sphere_c=(0.0, 0.0, 1.0), sphere_r=0.3):
    return [Plane((0.0, 0.0, 1.0), plane_z, (170, 170, 150)),
            Sphere(sphere_c, sphere_r, (210, 70, 50))]


def plane_sphere_frame(seed=20261203, noise=True, dropout=0.05, width=160,
                       height=120, intr=PLANE_SPHERE_INTR, pose=None, prims=None):
    """160x120 frame: plane 1.5 m away, 0.3 m sphere centred 1.0 m in front."""
    pose = np.eye(4) if pose is None else pose
    prims = plane_sphere_prims() if prims is None else prims
    return render(width, height, intr, pose, prims, seed, noise=noise, dropout=dropout)


# --- scene 2/3: room ------------------------------------------------------------
ROOM_INTR = (525.0, 525.0, 319.5, 239.5)
ROOM_HALF = 3.2          # walls at x, z = +-3.2 m
ROOM_FLOOR = 1.2         # y down: floor at y = +1.2, ceiling at y = -1.5
ROOM_CEIL = -1.5
ORBIT_R = 0.8
ORBIT_STEP_DEG = 1.2
ORBIT_START_DEG = 0.0


def room_prims(seed=20261204, n_boxes=6, n_spheres=4):
    """Axis-aligned room with seeded boxes (0.2-0.8 m edges) and spheres (r 0.1-0.4 m)."""
    prims = [
        Plane((1.0, 0.0, 0.0), ROOM_HALF, (200, 190, 170)),
        Plane((1.0, 0.0, 0.0), -ROOM_HALF, (190, 200, 170)),
        Plane((0.0, 0.0, 1.0), ROOM_HALF, (170, 190, 200)),
        Plane((0.0, 0.0, 1.0), -ROOM_HALF, (200, 170, 190)),
        Plane((0.0, 1.0, 0.0), ROOM_FLOOR, (120, 100, 80)),
        Plane((0.0, 1.0, 0.0), ROOM_CEIL, (230, 230, 230)),
    ]
    u = uniform(seed, 3, 256)
    k = 0

    def nxt():
        nonlocal k
        k += 1
        return float(u[k - 1])

    for _ in range(n_boxes):
        ex = [0.2 + 0.6 * nxt() for _ in range(3)]
        phi = 2 * math.pi * nxt()
        rho = 1.4 + 0.71 * max(ex[0], ex[2]) + 0.9 * nxt()
        cx_, cz_ = rho * math.sin(phi), rho * math.cos(phi)
        on_floor = nxt() < 0.6
        if on_floor:
            y1 = ROOM_FLOOR
            y0 = y1 - ex[1]
        else:
            y0 = -1.0 + 1.2 * nxt()
            y1 = y0 + ex[1]
        alb = tuple(int(40 + 200 * nxt()) for _ in range(3))
        prims.append(Box((cx_ - ex[0] / 2, y0, cz_ - ex[2] / 2),
                         (cx_ + ex[0] / 2, y1, cz_ + ex[2] / 2), alb))
    for _ in range(n_spheres):
        r = 0.1 + 0.3 * nxt()
        phi = 2 * math.pi * nxt()
        rho = 1.4 + r + 1.0 * nxt()
        y = -0.9 + 1.7 * nxt()
        alb = tuple(int(40 + 200 * nxt()) for _ in range(3))
        prims.append(Sphere((rho * math.sin(phi), y, rho * math.cos(phi)), r, alb))
    return prims


def orbit_pose(frame: int, seed=20261205):
    """Camera-to-world pose of frame f on the orbit: radius 0.8 m, 1.2 deg yaw per frame,
    looking outward, with a seeded smooth perturbation (about 1 cm, 0.5 deg)."""
    ph = uniform(seed, 5, 8) * 2 * math.pi
    f = float(frame)
    theta = math.radians(ORBIT_START_DEG + ORBIT_STEP_DEG * f)
    yaw = theta + math.radians(0.5) * math.sin(2 * math.pi * f / 97.0 + ph[0])
    pitch = math.radians(26.0) * math.sin(2 * math.pi * f / 100.0) + \
        math.radians(1.0) * math.sin(2 * math.pi * f / 131.0 + ph[1])
    roll = math.radians(0.5) * math.sin(2 * math.pi * f / 113.0 + ph[2])
    pos = np.array([ORBIT_R * math.sin(theta), 0.0, ORBIT_R * math.cos(theta)])
    pos = pos + 0.01 * np.array([math.sin(2 * math.pi * f / 89.0 + ph[3]),
                                 0.5 * math.sin(2 * math.pi * f / 71.0 + ph[4]),
                                 math.sin(2 * math.pi * f / 83.0 + ph[5])])
    return make_pose(rotation(yaw, pitch, roll), pos)


def room_frame(frame=0, seed=20261204, noise=True, dropout=0.05, width=640, height=480,
               intr=None, prims=None):
    """One frame of the room orbit. Intrinsics scale with width from the 640x480 camera."""
    if intr is None:
        s = width / 640.0
        intr = (525.0 * s, 525.0 * s, (width - 1) / 2.0, (height - 1) / 2.0)
    prims = room_prims(seed) if prims is None else prims
    return render(width, height, intr, orbit_pose(frame, seed + 1), prims,
                  seed * 1000 + frame, noise=noise, dropout=dropout)


def random_frame(seed, width=16, height=12, invalid=0.1, nonfinite=0.02):
    """Unstructured stress frame: random depths 0.2-3 m, random pose and intrinsics,
    with invalid (0, negative) and non-finite pixels. Exercises every branch of the
    per-voxel test rather than a realistic surface."""
    n = width * height
    u = uniform(seed, 21, n)
    depth = 0.2 + 2.8 * uniform(seed, 22, n)
    smooth = uniform(seed, 23, 1)[0] < 0.5
    if smooth:  # a tilted plane so neighbouring pixels agree and many voxels pass
        vv, uu = np.mgrid[0:height, 0:width]
        a, b, c = uniform(seed, 24, 3)
        depth = (0.6 + 1.5 * c + 0.02 * (a - 0.5) * uu.ravel() + 0.02 * (b - 0.5) * vv.ravel())
        depth = depth + 0.004 * normal(seed, 25, n)
    depth = np.where(u < invalid * 0.7, 0.0, depth)
    depth = np.where((u >= invalid * 0.7) & (u < invalid), -1.0, depth)
    bad = uniform(seed, 26, n) < nonfinite
    kinds = uniform(seed, 27, n)
    depth = np.where(bad & (kinds < 0.5), np.nan, depth)
    depth = np.where(bad & (kinds >= 0.5), np.inf, depth)
    r = uniform(seed, 28, 12)
    f = 10.0 + 30.0 * r[0]
    intr = (f, f * (0.9 + 0.2 * r[1]), (width - 1) / 2 + r[2] - 0.5, (height - 1) / 2 + r[3] - 0.5)
    R = rotation(2 * math.pi * r[4], 0.6 * (r[5] - 0.5), 0.6 * (r[6] - 0.5))
    t = (np.array(r[7:10]) - 0.5) * 4.0
    rgb = np.floor(uniform(seed, 29, n * 3) * 256).astype(np.uint8).reshape(height, width, 3)
    return Frame(depth=depth.astype(np.float32).reshape(height, width), rgb=rgb,
                 intr=np.asarray(intr, dtype=np.float32),
                 pose=make_pose(R, t).astype(np.float32))


# ----------------------------------------------------------------------------
# Workload configurations (the shapes of the paper's cells, Section 5)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class VolumeSpec:
    voxel_size: float
    truncation: float
    table_slots: int
    pool_blocks: int


PLANE_SPHERE_160 = VolumeSpec(0.01, 0.04, 1 << 16, 16384)
ROOM_640 = VolumeSpec(0.005, 0.02, 1 << 20, 1 << 18)
ROOM_ORBIT_300 = VolumeSpec(0.005, 0.02, 1 << 18, 1 << 18)   # load 0.035 -> 0.85 over the orbit


def session_mix(n_sessions=64, seed=20261206):
    """Batched-fusion sessions: resolution 160x120 / 320x240 / 640x480 chosen by seed,
    table 2^16 / 2^18 / 2^20 slots with pool = slots / 4, each its own room view."""
    u = uniform(seed, 31, n_sessions)
    res = [(160, 120, 1 << 16), (320, 240, 1 << 18), (640, 480, 1 << 20)]
    out = []
    for i in range(n_sessions):
        w, h, slots = res[min(2, int(u[i] * 3))]
        out.append(dict(session=i, width=w, height=h,
                        spec=VolumeSpec(0.005, 0.02, slots, slots // 4),
                        frame=int(uniform(seed, 32, n_sessions)[i] * 300)))
    return out
