"""Pins of the oracle's surface extraction (marching tetrahedra, readings E1-E4
in oracle/tsdf_oracle.cpp) against geometry, not against itself.

* one inside corner: six triangles (one per tetrahedron around the diagonal),
  vertices at the edge midpoints for values -1/2 and +1/2, normals pointing away
  from the inside corner;
* an unobserved corner removes its cube (E1);
* a linear field: linear interpolation of a linear function is exact, so every
  vertex lies on the plane, and every normal points to the positive side;
* a sphere's signed distance on a full grid: the surface is closed and
  consistently oriented (every directed edge once, its reverse once), has the
  topology of a sphere (V - E + F = 2), encloses 4/3 pi r^3 within the
  discretisation error, and every vertex is within a quarter voxel of the
  radius (the paper's correctness gate, Section 3.3);
* the same gate on a surface fused from a noise-free depth frame of the
  plane-and-sphere scene, where the surface faces the camera.
"""
import numpy as np
import pytest

import oracle
from paper_2608_08287_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def volume(v=0.1, tau=0.4):
    return oracle.OracleVolume(v, tau, 1 << 16, 1 << 16)


def normals(tris):
    return np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])


def test_one_inside_corner():
    ov = volume()
    for x in range(2):
        for y in range(2):
            for z in range(2):
                ov.set_voxel(x, y, z, -0.5 if (x, y, z) == (0, 0, 0) else 0.5)
    tris, cells = ov.extract()
    assert len(tris) == 6
    assert sorted(cells[:, 3].tolist()) == [0, 2, 4, 6, 8, 10]   # one per tetrahedron
    assert np.all(cells[:, :3] == 0)
    # vertices at the midpoints of the edges from (0.05, 0.05, 0.05)
    centre = np.array([0.05, 0.05, 0.05])
    for t in tris:
        for p in t:
            step = np.round((p - centre) / 0.05).astype(int)
            assert set(step.tolist()) <= {0, 1} and step.sum() >= 1
            assert np.allclose(p, centre + 0.05 * step)
    # normals point away from the inside corner
    mid = tris.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", normals(tris), mid - centre) > 0)


def test_one_outside_corner_flips_normals():
    ov = volume()
    for x in range(2):
        for y in range(2):
            for z in range(2):
                ov.set_voxel(x, y, z, 0.5 if (x, y, z) == (0, 0, 0) else -0.5)
    tris, _ = ov.extract()
    assert len(tris) == 6
    mid = tris.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", normals(tris), mid - 0.05) < 0)


def test_a_zero_corner_is_outside():
    """E3: inside means < 0. A corner at exactly 0 among positive corners makes
    no surface; among negative ones it is the lone outside corner, and its
    triangles meet at its own centre (t = 1 on every edge towards it)."""
    ov = volume()
    for x in range(2):
        for y in range(2):
            for z in range(2):
                ov.set_voxel(x, y, z, 0.0 if (x, y, z) == (0, 0, 0) else 0.5)
    assert len(ov.extract()[0]) == 0
    ov = volume()
    for x in range(2):
        for y in range(2):
            for z in range(2):
                ov.set_voxel(x, y, z, 0.0 if (x, y, z) == (1, 1, 1) else -0.5)
    tris, _ = ov.extract()
    assert len(tris) == 6
    assert np.allclose(tris, 0.15)


def test_unobserved_corner_removes_the_cube():
    ov = volume()
    for x in range(2):
        for y in range(2):
            for z in range(2):
                if (x, y, z) != (1, 1, 1):
                    ov.set_voxel(x, y, z, -0.5 if (x, y, z) == (0, 0, 0) else 0.5)
    assert len(ov.extract()[0]) == 0
    ov.set_voxel(1, 1, 1, 0.5, weight=3)   # a sum of 0.5 over 3 contributions
    assert len(ov.extract()[0]) == 6


def grid_volume(fn, n, v, lo=0):
    """Voxels [lo, lo+n)^3 set to fn(voxel centre); the centre uses the voxel
    size as the volume stores it (float32)."""
    ov = oracle.OracleVolume(v, 4 * v, 1 << 16, 1 << 16)
    v = float(np.float32(v))
    for x in range(lo, lo + n):
        for y in range(lo, lo + n):
            for z in range(lo, lo + n):
                p = (np.array([x, y, z]) + 0.5) * v
                ov.set_voxel(x, y, z, fn(p))
    return ov


def test_linear_field_is_reproduced_exactly():
    nrm = np.array([0.3, -0.5, 0.81])
    nrm /= np.linalg.norm(nrm)
    d = 0.05
    v = 0.01
    ov = grid_volume(lambda p: (p @ nrm - d) / 0.5, 16, v, lo=-8)
    tris, cells = ov.extract()
    assert len(tris) > 100
    assert np.max(np.abs(tris.reshape(-1, 3) @ nrm - d)) < 1e-12
    assert np.all(normals(tris) @ nrm > 0)


def _edges(tris):
    """Directed edges of every triangle, with vertices keyed by exact coordinates."""
    keys = {}
    ids = np.array([[keys.setdefault(tuple(p), len(keys)) for p in t] for t in tris])
    e = np.concatenate([ids[:, [0, 1]], ids[:, [1, 2]], ids[:, [2, 0]]])
    return ids, e, len(keys)


def test_sphere_surface_is_closed_oriented_and_within_a_quarter_voxel():
    v, r = 0.02, 0.3
    c = np.array([0.013, -0.007, 0.021])   # off the grid's symmetry
    tau = 4 * v
    ov = grid_volume(lambda p: float(np.clip((np.linalg.norm(p - c) - r) / tau, -1, 1)),
                     40, v, lo=-20)
    tris, cells = ov.extract()
    ids, e, nv = _edges(tris)
    # every directed edge exactly once, and its reverse exactly once
    directed = set(map(tuple, e.tolist()))
    assert len(directed) == len(e)
    assert all((b, a) in directed for a, b in directed)
    # Euler characteristic of a sphere
    undirected = {tuple(sorted(x)) for x in directed}
    assert nv - len(undirected) + len(tris) == 2
    # enclosed volume (divergence theorem) with outward normals
    vol = np.einsum("ij,ij->i", tris[:, 0], np.cross(tris[:, 1], tris[:, 2])).sum() / 6
    assert vol == pytest.approx(4 / 3 * np.pi * r ** 3, rel=0.01)
    # the paper's gate: every vertex within a quarter voxel of the radius
    dist = np.linalg.norm(tris.reshape(-1, 3) - c, axis=1)
    assert np.max(np.abs(dist - r)) <= v / 4


def facing_sphere_vertices(tris, c, r, v, max_angle_deg=60):
    """Vertices near the sphere whose surface normal is within max_angle of the
    direction back to the camera (at the origin)."""
    p = tris.reshape(-1, 3)
    d = np.linalg.norm(p - c, axis=1)
    near = np.abs(d - r) < 2 * v
    n = (p - c) / d[:, None]
    to_cam = -p / np.linalg.norm(p, axis=1)[:, None]
    facing = np.einsum("ij,ij->i", n, to_cam) > np.cos(np.radians(max_angle_deg))
    return p[near & facing], d[near & facing]


def test_fused_noise_free_sphere_meets_the_quarter_voxel_gate():
    f = synth.plane_sphere_frame(noise=False, dropout=0.0)
    spec = synth.PLANE_SPHERE_160
    ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                             spec.pool_blocks)
    assert ov.fuse_frame(f) == "OK"
    tris, _ = ov.extract()
    c, r = np.array([0.0, 0.0, 1.0]), 0.3
    p, d = facing_sphere_vertices(tris, c, r, spec.voxel_size)
    assert len(p) > 200
    assert np.max(np.abs(d - r)) <= spec.voxel_size / 4
    # the plane at z = 1.5 behind the sphere: vertices there lie on it
    plane = tris.reshape(-1, 3)
    plane = plane[np.abs(plane[:, 2] - 1.5) < 2 * spec.voxel_size]
    plane = plane[np.linalg.norm(plane[:, :2], axis=1) > 0.45]  # clear of the sphere's shadow
    assert len(plane) > 200
    assert np.max(np.abs(plane[:, 2] - 1.5)) <= spec.voxel_size / 4
