"""Pins for the CPU oracle: checks against things other than the oracle itself.

* a second, independent dense-grid statement of the frame (``brute_dense``);
* closed forms: a fronto-parallel plane seen from arbitrary poses, where the
  truncated projective distance of every accepted voxel centre is known exactly
  (paper Section 2, Section 4.1 on evaluating at the voxel centre);
* the paper's analytic gate: a sphere reproduced within a quarter voxel
  (Section 3.3 "Correctness", Section 4.1);
* invariants: each block once, no empty block, weights equal contribution counts
  (Section 2.2, "Both passes apply the same occlusion test");
* sums, not running means (Section 2.2);
* overflow is reported, never silent (Section 3.4, Section 7.2);
* the load-factor figures the paper prints (Section 7.2 table).
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle
from brute_dense import fma32, fuse_dense
from voxels import voxel_arrays, voxel_dict
from paper_2608_08287_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fuse(frame, v, tau, slots=1 << 16, pool=1 << 14, rgb=True):
    ov = oracle.OracleVolume(v, tau, slots, pool)
    st = ov.fuse_frame(frame, with_rgb=rgb)
    return ov, st


# ----------------------------------------------------------------------------
# the FMA emulation used by the dense brute force, against the C library
# ----------------------------------------------------------------------------
def test_fma32_emulation_matches_libm():
    libm = ctypes.CDLL(ctypes.util.find_library("m"))
    libm.fmaf.restype = ctypes.c_float
    libm.fmaf.argtypes = [ctypes.c_float] * 3
    rng = np.random.default_rng(7)
    a = rng.standard_normal(4000).astype(np.float32) * np.float32(3.0)
    b = rng.standard_normal(4000).astype(np.float32)
    c = -(a.astype(np.float64) * b).astype(np.float32)   # heavy cancellation cases
    c[::2] = rng.standard_normal(2000).astype(np.float32)
    # exact ties: a*b + c lands half-way between float32 neighbours
    a[:50] = np.float32(1.0) + np.float32(2.0 ** -12)
    b[:50] = np.float32(1.0) + np.float32(2.0 ** -12)
    c[:50] = np.float32(0.0)
    got = fma32(a, b, c)
    want = np.array([libm.fmaf(float(x), float(y), float(z)) for x, y, z in zip(a, b, c)],
                    dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # and it differs from the double-rounded separate multiply-add somewhere
    sep = (a * b) + c
    assert np.any(sep.view(np.uint32) != want.view(np.uint32))


# ----------------------------------------------------------------------------
# oracle == dense brute force on tiny frames
# ----------------------------------------------------------------------------
def _compare_with_brute(frame, v, tau):
    ov, st = _fuse(frame, v, tau, slots=1 << 14, pool=1 << 14)
    assert st == "OK"
    got = voxel_dict(*ov.export(double=True))
    want = fuse_dense(frame.depth, frame.intr, frame.pose, v, tau, rgb=frame.rgb)
    assert set(got) == set(want)
    for g, (w, t, r, gg, b) in want.items():
        o = got[g]
        assert o[1] == w, g
        assert abs(o[0] - t) <= 1e-12 and abs(o[2] - r) <= 1e-12
        assert abs(o[3] - gg) <= 1e-12 and abs(o[4] - b) <= 1e-12
    return ov.last_stats, len(want)


@pytest.mark.parametrize("seed", range(24))
def test_oracle_matches_dense_bruteforce_random(seed):
    f = synth.random_frame(1000 + seed, width=16, height=12)
    vt = [(0.05, 0.2), (0.1, 0.3), (0.03, 0.12), (0.02, 0.1)][seed % 4]
    stats, n = _compare_with_brute(f, *vt)
    assert stats["contributions"] >= n


@pytest.mark.parametrize("which", ["room", "plane_sphere"])
def test_oracle_matches_dense_bruteforce_scenes(which):
    if which == "room":
        f = synth.room_frame(17, width=40, height=30)
        v, tau = 0.05, 0.2
    else:
        f = synth.plane_sphere_frame(width=40, height=30, intr=(35.0, 35.0, 20.0, 15.0))
        v, tau = 0.02, 0.08
    stats, n = _compare_with_brute(f, v, tau)
    assert n > 200  # the frame actually exercises accumulation


def test_fp_contract_exact_binary_ties():
    """Exact binary geometry puts samples and projections on voxel and pixel boundaries;
    every floor() decision must agree between the two statements."""
    H = W = 8
    vals = (np.arange(H * W) % 13 + 20).astype(np.float32) / np.float32(16.0)
    depth = vals.reshape(H, W)
    depth[3, 3] = np.nextafter(depth[3, 3], np.float32(9))
    depth[4, 5] = np.nextafter(depth[4, 5], np.float32(0))
    intr = np.array([8.0, 8.0, 3.5, 3.5], dtype=np.float32)
    for pose in (np.eye(4), synth.make_pose(synth.rotation(math.pi / 2), [0.25, -0.5, 0.125])):
        fr = synth.Frame(depth=depth, rgb=np.full((H, W, 3), 100, np.uint8), intr=intr,
                         pose=pose.astype(np.float32))
        _compare_with_brute(fr, 0.125, 0.5)


def test_fp_contract_ulp_neighbourhood():
    """Depths one to three ulps either side of voxel boundaries (v = 1 cm is inexact)."""
    H, W = 6, 7
    base = np.float32(1.23)
    d = np.empty(H * W, dtype=np.float32)
    for i in range(H * W):
        x = base + np.float32(0.01) * np.float32(i % 5)
        for _ in range(i % 7 - 3):
            x = np.nextafter(x, np.float32(9))
        for _ in range(3 - i % 7):
            x = np.nextafter(x, np.float32(0))
        d[i] = x
    fr = synth.Frame(depth=d.reshape(H, W), rgb=np.zeros((H, W, 3), np.uint8),
                     intr=np.array([6.0, 6.0, 3.0, 2.5], np.float32),
                     pose=np.eye(4, dtype=np.float32))
    _compare_with_brute(fr, 0.01, 0.04)


# ----------------------------------------------------------------------------
# closed form: fronto-parallel plane, arbitrary camera pose
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("pose_id", range(4))
def test_plane_closed_form(pose_id):
    Z = np.float32(1.3)
    W, H = 64, 48
    v, tau = 0.01, 0.04
    if pose_id == 0:
        pose = np.eye(4)
    else:
        r = synth.uniform(500 + pose_id, 1, 6)
        pose = synth.make_pose(synth.rotation(2 * math.pi * r[0], r[1] - 0.5, r[2] - 0.5),
                               (r[3:6] - 0.5) * 3.0)
    pose = pose.astype(np.float32)
    fr = synth.Frame(depth=np.full((H, W), Z, np.float32), rgb=np.zeros((H, W, 3), np.uint8),
                     intr=np.array([60.0, 60.0, 31.5, 23.5], np.float32), pose=pose)
    ov, st = _fuse(fr, v, tau)
    assert st == "OK"
    g, vals = voxel_arrays(*ov.export(double=True))
    assert len(g) > 1000
    P = pose.astype(np.float64)
    cw = (g.astype(np.float64) + 0.5) * v
    zc = (cw - P[:3, 3]) @ P[:3, 2]          # camera z = R^T (c - t), third component
    want = np.clip((float(Z) - zc) / tau, -1.0, 1.0)
    # float32 rounding of the centre (|c| < 4 m, a few roundings) bounds the error:
    # about 1e-6 m in z_c, i.e. 2.5e-5 in units of tau; 5e-5 leaves margin.
    assert np.max(np.abs(vals[:, 0] - want)) < 5e-5
    # accepted voxels are never more than tau behind the surface (occlusion test)
    assert np.all(zc <= float(Z) + tau + 1e-6)
    # and they lie within the truncation band plus one voxel diagonal
    assert np.all(np.abs(zc - float(Z)) <= tau + v * math.sqrt(3) + 1e-6)
    # both sides of the surface are present
    assert (want > 0.5).any() and (want < -0.5).any()


def test_colour_means_closed_form():
    """Reading R4: a voxel's colour is the mean over the points that reached it
    of their own pixel's 8-bit colour, divided by 255. The left half of the
    image is colour A, the right half colour B, so every voxel's mean is
    A/255 + a (B - A)/255 with one mixing fraction a = n_B / w shared by the
    three channels, n_B a whole number of points; voxels reached from one half
    only carry exactly that colour."""
    H, W, Z, split = 48, 64, np.float32(1.3), 35
    A = np.array([10, 20, 30])
    B = np.array([200, 150, 100])
    rgb = np.empty((H, W, 3), np.uint8)
    rgb[:, :split] = A
    rgb[:, split:] = B
    # about 4.6 pixels per 1 cm voxel, and a split inside a voxel: mixed voxels
    fr = synth.Frame(depth=np.full((H, W), Z, np.float32), rgb=rgb,
                     intr=np.array([600.0, 600.0, 31.5, 23.5], np.float32),
                     pose=np.eye(4, dtype=np.float32))
    ov, st = _fuse(fr, 0.01, 0.04)
    assert st == "OK"
    g, vals = voxel_arrays(*ov.export(double=True))
    w = vals[:, 1]
    col = vals[:, 2:5] * 255.0
    alpha = (col - A) / (B - A)                      # per channel
    assert np.allclose(alpha, alpha[:, :1], atol=1e-9)
    nb = alpha[:, 0] * w
    assert np.allclose(nb, np.round(nb), atol=1e-6)
    assert np.all((np.round(nb) >= 0) & (np.round(nb) <= w))
    pure_a, pure_b = np.isclose(alpha[:, 0], 0), np.isclose(alpha[:, 0], 1)
    assert pure_a.sum() > 100 and pure_b.sum() > 100 and (~pure_a & ~pure_b).any()
    # the pure voxels lie on their own side of the split, a voxel at most away
    x_split = (split - 0.5 - 31.5) / 600.0 * 1.3
    cx = (g[:, 0] + 0.5) * 0.01
    assert np.all(cx[pure_a] < x_split + 0.01) and np.all(cx[pure_b] > x_split - 0.01)


# ----------------------------------------------------------------------------
# the paper's analytic gate: sphere within a quarter voxel
# ----------------------------------------------------------------------------
def test_sphere_within_quarter_voxel():
    C = np.array([0.0, 0.0, 1.0])
    r = 0.3
    v, tau = 0.01, 0.04
    prims = [synth.Sphere(tuple(C), r)]
    f = synth.plane_sphere_frame(noise=False, dropout=0.0, width=320, height=240,
                                 intr=(280.0, 280.0, 160.0, 120.0), prims=prims)
    ov, st = _fuse(f, v, tau)
    assert st == "OK"
    g, vals = voxel_arrays(*ov.export(double=True))
    tsdf = {tuple(x): val[0] for x, val in zip(g.tolist(), vals)}
    errs = []
    for (x, y, z), t0 in tsdf.items():
        t1 = tsdf.get((x, y, z + 1))
        if t1 is None or not (t0 > 0.0 >= t1):
            continue
        za = (z + 0.5) * v
        z0 = za + t0 / (t0 - t1) * v
        p = np.array([(x + 0.5) * v, (y + 0.5) * v, z0])
        nrm = (p - C) / np.linalg.norm(p - C)
        view = p / np.linalg.norm(p)
        if -nrm @ view < math.cos(math.radians(60)):
            continue
        errs.append(abs(np.linalg.norm(p - C) - r))
    assert len(errs) > 500
    assert max(errs) <= v / 4, max(errs)


# ----------------------------------------------------------------------------
# invariants on the workload frames
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["plane_sphere_160", "room_640"])
def test_invariants(which):
    if which == "plane_sphere_160":
        f, spec = synth.plane_sphere_frame(), synth.PLANE_SPHERE_160
    else:
        f, spec = synth.room_frame(0), synth.ROOM_640
    ov, st = _fuse(f, spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    assert st == "OK"
    s = ov.last_stats
    coords, vox = ov.export()
    M = int(round(spec.truncation / spec.voxel_size))
    assert s["points"] == f.valid_points
    assert s["samples"] == s["points"] * (2 * M + 1)
    assert len({tuple(c) for c in coords.tolist()}) == len(coords)           # each key once
    assert np.all((vox[:, 1, :] > 0).any(axis=1))                            # no empty block
    assert int(vox[:, 1, :].sum()) == s["contributions"]                     # weights = count
    assert int((vox[:, 1, :] > 0).sum()) == s["unique_voxels"]
    assert len(coords) == s["unique_blocks"] == s["new_blocks"] == ov.block_count()
    w = vox[:, 1, :]
    assert np.all(np.abs(vox[:, 0, :]) <= 1.0)
    assert np.all((vox[:, 2:, :] >= 0) & (vox[:, 2:, :] <= 1.0))
    assert np.all(w == np.floor(w))


def test_sums_not_running_means():
    spec = synth.PLANE_SPHERE_160
    fa = synth.plane_sphere_frame(seed=1)
    fb = synth.plane_sphere_frame(seed=2)
    both = oracle.OracleVolume(spec.voxel_size, spec.truncation, 1 << 16, 1 << 14)
    assert both.fuse_frame(fa) == "OK" and both.fuse_frame(fb) == "OK"
    a, _ = _fuse(fa, spec.voxel_size, spec.truncation)
    b, _ = _fuse(fb, spec.voxel_size, spec.truncation)
    da = voxel_dict(*a.export(double=True))
    db = voxel_dict(*b.export(double=True))
    dab = voxel_dict(*both.export(double=True))
    assert set(dab) == set(da) | set(db)
    for g, val in dab.items():
        wa = da.get(g, (0.0, 0.0))[1]
        wb = db.get(g, (0.0, 0.0))[1]
        assert val[1] == wa + wb
        ta = da[g][0] if g in da else 0.0
        tb = db[g][0] if g in db else 0.0
        assert abs(val[0] - (wa * ta + wb * tb) / (wa + wb)) < 1e-12


def test_overflow_reported_and_poisons():
    f = synth.plane_sphere_frame()
    spec = synth.PLANE_SPHERE_160
    ov, st = _fuse(f, spec.voxel_size, spec.truncation)
    D = ov.block_count()
    assert st == "OK" and D > 100
    ok, st = _fuse(f, spec.voxel_size, spec.truncation, pool=D)
    assert st == "OK" and ok.block_count() == D
    bad, st = _fuse(f, spec.voxel_size, spec.truncation, pool=D - 1)
    assert st == "POOL_FULL"
    assert bad.block_count() == D - 1
    assert bad.last_stats["over_pool"] == 1
    assert bad.fuse_frame(f) == "POISONED"
    bad.reset()
    assert bad.block_count() == 0
    tiny, st = _fuse(f, spec.voxel_size, spec.truncation, slots=64, pool=16)
    assert st == "POOL_FULL" and tiny.block_count() == 16
    # with the pool as large as the table, the table is what runs out
    full, st = _fuse(f, spec.voxel_size, spec.truncation, slots=16, pool=16)
    assert st == "TABLE_FULL" and full.block_count() == 16


def test_rejects_bad_parameters():
    for args in [(0.0, 0.04, 1024, 64), (0.01, 0.005, 1024, 64), (0.01, 0.04, 1000, 64),
                 (0.01, 0.04, 1024, 2048), (0.01, 0.04, 1024, 0)]:
        with pytest.raises(ValueError):
            oracle.OracleVolume(*args)


def test_paper_load_factor_table():
    """Section 7.2 prints load factors for a 1,160-block sphere; blocks / slots with
    slots = 2^16 ... 2^12 reproduces every printed value (the definition the orbit
    workload's load factor uses)."""
    rows = []
    with open(os.path.join(GOLDEN, "paper_load_factors.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                cell, load, blocks = line.split()
                rows.append((cell, float(load), int(blocks)))
    slots = {"lf-sparse": 1 << 16, "base": 1 << 15, "lf-lo": 1 << 14, "lf-mid": 1 << 13,
             "lf-hi": 1 << 12}
    for cell, load, blocks in rows:
        assert round(blocks / slots[cell], 3) == load, cell
