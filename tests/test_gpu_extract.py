"""Surface extraction on the GPU (tsdf_extract_mesh) against the oracle's
marching tetrahedra on the same fused frames.

Each triangle is named by its cell record {gx, gy, gz, 2*tetrahedron + k},
so the two meshes are compared as sets of names, exactly. A corner's sign can
legitimately differ between the two only where its mean tsdf is within the
fusion tolerance (1e-5) of zero, because the GPU sums in float32 in another
order; the tetrahedra with such a corner are left out of the exact
comparison (they are counted, and must be rare). For the rest the vertices
must agree within the error those same means allow: a vertex sits at
t = v_a / (v_a - v_b) along its edge, so a mean error e moves it by at most
e / |v_a - v_b| of the edge, plus float32 rounding of the coordinates.
The sphere gate of the paper (Section 3.3: the sphere within a quarter voxel)
is checked on the GPU's own mesh.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2608_08287_gb300 import synth, tsdf
from test_gpu_parity import to_dev
from test_oracle_extract import facing_sphere_vertices

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-5        # fusion parity tolerance on tsdf means
AMBIGUOUS = 2e-5       # corners this close to zero may change sign
TETS = [(0, 1, 3, 7), (0, 1, 7, 5), (0, 2, 7, 3), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 7, 6)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_08287_gb300.build import build_library
    build_library()
    oracle.build()
    torch.cuda.set_device(0)


TET_OFFSETS = np.array([[[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in t] for t in TETS])


def _pack(b):
    b = b.astype(np.int64) + (1 << 20)
    return (b[..., 0] << 42) | (b[..., 1] << 21) | b[..., 2]


class Means:
    """The oracle's mean tsdf per voxel, looked up in bulk (NaN where unobserved)."""

    def __init__(self, ov):
        coords, vox = ov.export(double=True)
        keys = _pack(coords)
        order = np.argsort(keys)
        self.keys = keys[order]
        self.tsdf = vox[order, 0]
        self.weight = vox[order, 1]

    def corners(self, cells):
        """(n, 4) means at the four corners of each cell's tetrahedron."""
        g = cells[:, None, :3].astype(np.int64) + TET_OFFSETS[cells[:, 3] // 2]
        key = _pack(g >> 3)
        l = (g[..., 0] & 7) + 8 * (g[..., 1] & 7) + 64 * (g[..., 2] & 7)
        pos = np.minimum(np.searchsorted(self.keys, key), len(self.keys) - 1)
        found = self.keys[pos] == key
        val = self.tsdf[pos, l]
        ok = found & (self.weight[pos, l] > 0)
        return np.where(ok, val, np.nan)


def _rows(cells):
    return cells.astype(np.int64).view([("", np.int64)] * 4).ravel()


def compare(gpu, ora, means, voxel):
    gt, gc = gpu
    ot, oc = ora
    gr, orr = _rows(gc), _rows(oc)
    assert len(np.unique(gr)) == len(gr) and len(np.unique(orr)) == len(orr)  # unique names
    vg, vo = means.corners(gc), means.corners(oc)
    assert not np.isnan(vg).any() and not np.isnan(vo).any()   # only observed cubes
    amb_g = np.min(np.abs(vg), axis=1) <= AMBIGUOUS
    amb_o = np.min(np.abs(vo), axis=1) <= AMBIGUOUS
    keep_g, keep_o = gr[~amb_g], orr[~amb_o]
    # the unambiguous names are the same set
    assert len(keep_g) == len(keep_o)
    sg, so = np.argsort(keep_g), np.argsort(keep_o)
    assert np.array_equal(keep_g[sg], keep_o[so])
    # matched vertices within the error the means allow
    tg = gt[~amb_g][sg].astype(np.float64)
    to = ot[~amb_o][so]
    v = vo[~amb_o][so]
    neg = v < 0
    span = np.full(len(v), np.inf)
    for a in range(4):
        for b in range(4):
            cross = neg[:, a] != neg[:, b]
            span = np.where(cross, np.minimum(span, np.abs(v[:, a] - v[:, b])), span)
    bound = np.sqrt(3) * voxel * 2 * MEAN_TOL / span + 4e-6
    err = np.max(np.abs(tg - to).reshape(len(tg), -1), axis=1)
    assert np.all(err <= bound), (np.max(err - bound), int(np.argmax(err - bound)))
    ambiguous = int(amb_o.sum())
    assert ambiguous <= 1e-3 * max(1, len(oc)), ambiguous
    return len(oc), ambiguous, float(err.max()) if len(err) else 0.0


def fuse(frames, spec, **opts):
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    for k, x in opts.items():
        assert gv.set_option(k, x) == "OK"
    ov = oracle.OracleVolume(spec.voxel_size, spec.truncation, spec.table_slots,
                             spec.pool_blocks)
    for f in frames:
        d, c = to_dev(f)
        assert gv.fuse(d, f.intr, f.pose, c) == ov.fuse_frame(f) == "OK"
    return gv, ov


@pytest.mark.parametrize("slot_index", [0, 1])
def test_plane_sphere_mesh_matches_oracle(slot_index):
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 16, 1 << 16)
    gv, ov = fuse([synth.plane_sphere_frame()], spec, slot_index=slot_index)
    tris, cells, timing = gv.extract_mesh()
    n, amb, worst = compare((tris, cells), ov.extract(), Means(ov), spec.voxel_size)
    assert n > 5000
    assert timing["compute_ms"] > 0 and timing["d2h_bytes"] == n * 52


def test_room_orbit_mesh_matches_oracle():
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 16, 1 << 15)
    frames = [synth.room_frame(k, width=320, height=240) for k in (0, 20, 40)]
    gv, ov = fuse(frames, spec)
    tris, cells, _ = gv.extract_mesh()
    n, amb, worst = compare((tris, cells), ov.extract(), Means(ov), spec.voxel_size)
    assert n > 50000


def test_gpu_sphere_meets_the_quarter_voxel_gate():
    spec = synth.PLANE_SPHERE_160
    f = synth.plane_sphere_frame(noise=False, dropout=0.0)
    gv = tsdf.Volume(spec.voxel_size, spec.truncation, spec.table_slots, spec.pool_blocks)
    d, c = to_dev(f)
    assert gv.fuse(d, f.intr, f.pose, c) == "OK"
    tris, _, _ = gv.extract_mesh(cells=False)
    p, dist = facing_sphere_vertices(tris.astype(np.float64), np.array([0.0, 0.0, 1.0]), 0.3,
                                     spec.voxel_size)
    assert len(p) > 200
    assert np.max(np.abs(dist - 0.3)) <= spec.voxel_size / 4


def test_capacity_contract_and_device_output():
    spec = synth.VolumeSpec(0.01, 0.04, 1 << 16, 1 << 16)
    gv, ov = fuse([synth.plane_sphere_frame(seed=9)], spec)
    tris, cells, _ = gv.extract_mesh()
    n = len(tris)
    # too small a host buffer: nothing copied, the count reported
    out = np.zeros((10, 9), dtype=np.float32)
    m = tsdf.ctypes.c_uint32()
    st = tsdf._st(tsdf.lib().tsdf_extract_mesh(gv.handle, out.ctypes.data, None, 10,
                                               tsdf.ctypes.byref(m), None, None))
    assert st == "INVALID_ARG" and m.value == n and not out.any()
    # device output, with a capacity short by 100: the first n - 100 are written
    cap = n - 100
    dt = torch.zeros((cap, 9), dtype=torch.float32, device="cuda")
    dc = torch.full((cap, 4), -7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert tsdf.tsdf_extract_mesh_async(gv.handle, dt, dc, cap, cnt) == "OK"
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    got = {tuple(x) for x in dc.cpu().numpy().tolist()}
    assert len(got) == cap and got <= {tuple(x) for x in cells.tolist()}
    # an empty volume has no surface
    assert gv.reset() == "OK"
    assert len(gv.extract_mesh()[0]) == 0
